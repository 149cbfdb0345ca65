"""Pins of the oracle's near-boundary flags (oracle.exact.flags_of) and of the
brute-force ragged oracle's indexing (oracle.ragged), to things other than
themselves.

The flags mark where a correct floating-point kernel may legitimately decide
differently from the exact answer, and every parity test leaves flagged arcs
out of its exact comparisons, so they are pinned here on inputs whose
distance to each boundary is known without the oracle:

* near tangency (whether the circles meet, Sec. 2): arcs in the plane of
  (a, 0, b) and the y-axis, x1 = (a, Y, b), x2 = (a, -Y, b), against z0 = 1/2.
  Then n = (2Yb, 0, -2aY), |n_xy|^2 = 4 Y^2 b^2, |n|^2 = 4 Y^2 (a^2 + b^2) and
  s^2 = |n_xy|^2 - |n|^2 / 4 = Y^2 (3 b^2 - a^2). The integer solutions of
  a^2 - 3 b^2 = -2 (s^2 > 0) and a^2 - 3 b^2 = 1 (s^2 < 0), two Pell-type
  families, give |s^2| / |n_xy|^2 = 1 / (2 b^2) and 1 / (4 b^2) exactly: the
  flag must be set iff that is <= 2^-96;
* near an endpoint (whether the candidate lies between the endpoints, Sec. 2):
  the candidate's distance from the endpoint is found by bisection along the
  great circle at 80 digits (no Eq. 2.2), and the flag must be set iff the
  sine of that angle is < 2^-40, for candidates at about 2^-41 and 2^-39, in
  both output slots;
* tiny normals: x2 = x1 + 2^-k e with exactly representable inputs;
* ordinary arcs (the uniform, stress and mixed workloads) carry almost no
  flag, so the parity tests that skip flagged arcs still test nearly all;
* planted mistakes (the tangency threshold at 2^-40 or 2^-120, the endpoint
  threshold moved, the slot sign dropped from the endpoint test) each fail
  one of these pins.

The ragged brute force is pinned on a two-mesh toy whose hits are listed by
hand from closed forms (meridian and equator arcs), with a latitude of the
other mesh that would hit the edge if it were (wrongly) applied.
"""
import inspect
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

from oracle import exact
from oracle import ragged as oracle_ragged
from paper_2510_09892_gb300 import workloads as W


# --------------------------------------------------------- near tangency --
def _pell(start, bmax=1 << 53):
    """Solutions (a, b) of a^2 - 3 b^2 = const from `start`, by (a, b) -> (2a + 3b, a + 2b)."""
    a, b = start
    out = []
    while a < bmax and b < bmax:
        out.append((a, b))
        a, b = 2 * a + 3 * b, a + 2 * b
    return out


def _tangent_cases():
    cases = []
    for (a, b) in _pell((1, 1)):          # a^2 - 3 b^2 = -2: s^2 > 0, gap 1 / (2 b^2)
        assert a * a - 3 * b * b == -2
        cases.append((a, b, +1, math.log2(2 * b * b)))
    for (a, b) in _pell((2, 1)):          # a^2 - 3 b^2 = 1: s^2 < 0, gap 1 / (4 b^2)
        assert a * a - 3 * b * b == 1
        cases.append((a, b, -1, math.log2(4 * b * b)))
    return cases                          # (a, b, sign of s^2, -log2 of the gap)


def _check_tangent_flags():
    seen = {True: 0, False: 0}
    for a, b, sgn, e in _tangent_cases():
        x1 = (float(a), float(b), float(b))
        x2 = (float(a), -float(b), float(b))
        assert int(x1[0]) == a and int(x1[2]) == b  # inputs exact
        r = exact.intersect(x1, x2, 0.5)
        want = e >= exact_threshold_log2()
        got = bool(r.flags & exact.FLAG_NEAR_TANGENT)
        assert got == want, (a, b, e, r.flags)
        if e >= 20:
            # the circles meet iff s^2 > 0; the candidates then lie within about
            # 2^-10 of the apex, well inside the arc (|y| <= 0.4 on it)
            assert r.count == (2 if sgn > 0 else 0), (a, b, r.count)
        if 80 <= e <= 110:
            seen[want] += 1
    assert seen[True] >= 2 and seen[False] >= 2, seen


def exact_threshold_log2():
    """The threshold the paper's error analysis justifies: the computed s^2
    carries an error of order u^2 |n|^2 (Sec. 6.1), 2^-106 relative, so its
    sign is trusted above 2^-96 |n_xy|^2. Stated here, not read from the oracle."""
    return 96


def test_near_tangent_flag_threshold():
    _check_tangent_flags()


@pytest.mark.parametrize("planted", [40, 90, 100, 120])
def test_planted_tangent_threshold_is_caught(monkeypatch, planted):
    monkeypatch.setattr(exact, "TANGENT_LOG2", planted)
    with pytest.raises(AssertionError):
        _check_tangent_flags()


# --------------------------------------------------------- near an endpoint --
def _dvec(v):
    return [Decimal(float(c)) for c in v]


def _cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def _norm(v):
    return (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]).sqrt()


def _endpoint_distance(x1, x2, z0, end):
    """Sine of the angle between endpoint `end` and the point of the great
    circle through x1, x2 at height z0 next to it: bisection at 80 digits on
    the normalised chord (1 - t) x1 + t x2, extended past the endpoint, over
    t in t_end +- 2^-16 where the height is monotone. Returns (sine, point)."""
    getcontext().prec = 80
    X1, X2, Z0 = _dvec(x1), _dvec(x2), Decimal(float(z0))

    def point(t):
        c = [(1 - t) * p + t * q for p, q in zip(X1, X2)]
        n = _norm(c)
        return [v / n for v in c]

    t0 = Decimal(end)
    lo, hi = t0 - Decimal(2) ** -16, t0 + Decimal(2) ** -16
    flo = point(lo)[2] - Z0
    fhi = point(hi)[2] - Z0
    assert (flo > 0) != (fhi > 0), "height not bracketed"
    for _ in range(230):
        mid = (lo + hi) / 2
        fm = point(mid)[2] - Z0
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    P = point((lo + hi) / 2)
    E = X1 if end == 0 else X2
    return _norm(_cross(E, P)) / _norm(E), P


def _endpoint_cases(n=160, seed=5):
    """Arcs of length U(0.3, 1.2) whose latitude passes about 2^-41 or 2^-39
    rad inside or outside one endpoint, where the height changes by >= 0.3 per
    radian along the arc."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        a = rng.standard_normal(3)
        a /= np.linalg.norm(a)
        b = rng.standard_normal(3)
        b -= b.dot(a) * a
        b /= np.linalg.norm(b)
        L = rng.uniform(0.3, 1.2)
        end = int(rng.integers(2))
        te = 0.0 if end == 0 else L
        if abs(-math.sin(te) * a[2] + math.cos(te) * b[2]) < 0.3:
            continue
        d = (2.0 ** -41 if len(out) % 2 == 0 else 2.0 ** -39) * rng.uniform(0.9, 1.1)
        d *= 1 if rng.random() < 0.5 else -1
        t = te + (d if end == 0 else -d)
        z0 = math.cos(t) * a[2] + math.sin(t) * b[2]
        x2 = math.cos(L) * a + math.sin(L) * b
        out.append((tuple(a), tuple(x2), float(z0), end))
    return out


def _check_endpoint_flags():
    near_slots = set()
    sides = {True: 0, False: 0}
    for x1, x2, z0, end in _endpoint_cases():
        sine, P = _endpoint_distance(x1, x2, z0, end)
        want = sine < Decimal(2) ** -40
        r = exact.intersect(x1, x2, z0)
        assert r.flags & ~exact.FLAG_NEAR_ENDPOINT == 0, r.flags
        got = bool(r.flags & exact.FLAG_NEAR_ENDPOINT)
        assert got == want, (x1, x2, z0, end, float(sine))
        sides[want] += 1
        if want:
            ex = exact.setup(x1, x2, z0)
            for slot, sigma in enumerate((1, -1)):
                c = exact.candidate_point(ex, sigma)
                if max(abs(Decimal(c[k]) - P[k]) for k in range(2)) < Decimal(2) ** -45:
                    near_slots.add(slot)
    assert sides[True] >= 40 and sides[False] >= 40, sides
    assert near_slots == {0, 1}, near_slots


def test_near_endpoint_flag_threshold():
    _check_endpoint_flags()


def _flags_without_slot_sign():
    """flags_of with the slot's sign dropped from the endpoint test (a planted mistake)."""
    src = inspect.getsource(exact.flags_of)
    bad = src.replace("sigma * _dot", "_dot")
    assert bad != src
    ns = dict(vars(exact))
    exec(compile(bad, "<planted>", "exec"), ns)
    return ns["flags_of"]


@pytest.mark.parametrize("planted", ["no_slot_sign", "log2_38", "log2_42"])
def test_planted_endpoint_mistakes_are_caught(monkeypatch, planted):
    if planted == "no_slot_sign":
        monkeypatch.setattr(exact, "flags_of", _flags_without_slot_sign())
    else:
        monkeypatch.setattr(exact, "ENDPOINT_LOG2", int(planted[-2:]))
    with pytest.raises(AssertionError):
        _check_endpoint_flags()


# ------------------------------------------------------------ tiny normals --
def test_tiny_normal_flag():
    x1 = (1.0, 0.0, 0.0)
    for k in (190, 199, 201, 230):
        x2 = (1.0, 2.0 ** -k, 0.0)  # n = (0, 0, 2^-k) exactly, |x1| = 1, |x2| = 1 + O(2^-2k)
        r = exact.intersect(x1, x2, 0.25)
        assert bool(r.flags & exact.FLAG_TINY_NORMAL) == (k > 200), k


# ------------------------------------------------------------ ordinary arcs --
def _check_ordinary_unflagged():
    A, B, z = W.uniform_arcs(3000, seed=21)
    _, _, f = exact.intersect_batch(A, B, z)
    assert np.count_nonzero(f) == 0
    A, B, z = W.stress_arcs(4000, seed=22)
    _, _, f = exact.intersect_batch(A, B, z)
    assert np.count_nonzero(f & exact.FLAG_NEAR_TANGENT) == 0
    assert np.count_nonzero(f) <= 4  # <= 0.1 %: near-endpoint short arcs only
    A, B, z = W.mixed_chunk(5, size=3000)
    _, _, f = exact.intersect_batch(A, B, z)
    assert np.count_nonzero(f) <= 3


def test_ordinary_arcs_are_unflagged():
    _check_ordinary_unflagged()


def test_planted_tangent_40_flags_ordinary_arcs(monkeypatch):
    monkeypatch.setattr(exact, "TANGENT_LOG2", 40)
    with pytest.raises(AssertionError):
        _check_ordinary_unflagged()


def test_near_boundary_workload_spans_both_sides():
    """The near-boundary generator places arcs on both sides of each flag's
    threshold: its tangency gaps and endpoint distances are checked here
    against their construction, on a small sample."""
    A, B, z, k = W.near_boundary_arcs(400, seed=3, return_class=True)
    _, _, f = exact.intersect_batch(A, B, z)
    names = [c for c, _ in W.NEAR_CLASSES]
    tan = np.isin(k, [names.index("tangent"), names.index("tangent_rotated")])
    ep = k == names.index("endpoint_offset")
    ez = k == names.index("endpoint_z")
    assert 0.1 < np.mean(f[tan] & exact.FLAG_NEAR_TANGENT > 0) < 0.6
    assert 0.15 < np.mean(f[ep] & exact.FLAG_NEAR_ENDPOINT > 0) < 0.55
    assert np.all(f[ez] & exact.FLAG_NEAR_ENDPOINT)


# ------------------------------------------------------------- ragged toy --
def test_ragged_oracle_two_mesh_toy():
    """Mesh 0: a meridian quarter from (1,0,0) up to the pole and a meridian
    quarter from (0,1,0) down to the south pole, latitudes {-0.5, 0.5}.
    Mesh 1: an equator arc from (1,0,0) to (0,1,0) and a meridian quarter
    from (0,-1,0) up to the pole, latitudes {0, 0.6}.

    For a meridian arc through (c, d, 0) the candidates at height z0 are
    +-sqrt(1 - z0^2) (c, d) (Eq. 2.2 with n_z = 0); slot 0 takes the sign of
    -n_y for n = x1 x x2 ... as listed: edge 0 (n = (0,-1,0)) hits z = 0.5 in
    slot 0 at x = sqrt(0.75); edge 1 (n = (-1,0,0)) hits z = -0.5 at
    y = sqrt(0.75), slot 1; edge 2 lies on the equator: z = 0 is coincident
    (degenerate), 0.6 is missed; edge 3 (n = (-1,0,0)) hits z = 0.6 at
    y = -0.8 in slot 0 and z = 0 at y = -1 in slot 0. Mesh 1's latitude 0.6
    would hit edge 0 if it were applied there."""
    A = np.array([[1.0, 0, 0], [0, 1.0, 0], [1.0, 0, 0], [0, -1.0, 0]])
    B = np.array([[0, 0, 1.0], [0, 0, -1.0], [0, 1.0, 0], [0, 0, 1.0]])
    eo = np.array([0, 2, 4])
    lat = np.array([-0.5, 0.5, 0.0, 0.6])
    lo = np.array([0, 2, 4])
    recs, flagged, degen = oracle_ragged.intersect_ragged(A, B, eo, lat, lo)
    s = math.sqrt(0.75)
    want = {(0, 1, 0, s, 0.0), (1, 0, 1, 0.0, s), (3, 3, 0, 0.0, -0.8), (3, 2, 0, 0.0, -1.0)}
    got = {(e, k, r, x, y) for e, k, r, x, y in recs}
    assert len(recs) == len(got)
    assert {g[:3] for g in got} == {w[:3] for w in want}, sorted(got)
    for e, k, r, x, y in got:
        w = next(v for v in want if v[:3] == (e, k, r))
        assert abs(x - w[3]) <= 2.3e-16 and abs(y - w[4]) <= 2.3e-16, (e, k, r, x, y)
    assert degen == {(2, 2)}
    # an edge subset keeps global indices
    recs3, _, _ = oracle_ragged.intersect_ragged(A, B, eo, lat, lo, edges=[3])
    assert {r[:3] for r in recs3} == {(3, 3, 0), (3, 2, 0)}
