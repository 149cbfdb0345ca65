"""Pins of the step-by-step FP64 reference (oracle/accux_ref.c via oracle/steps.py).

Each building block is checked against exact rational arithmetic and the
error bound the paper states for it (Sec. 5, supplement S2), and AccuX as a
whole against the exact oracle and the bound of Sec. 6.2. The literal AccuDOP
of Algorithm 4 ('+' between r1 and r2) is shown to break its own bound, which
is why the reference (and the CUDA path) read it as r1 - r2.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import exact, steps
from paper_2510_09892_gb300 import workloads as W

U = 2.0 ** -53
Uf = Fr(1, 1 << 53)


def _rand(rng, n, lo=-1.0, hi=1.0):
    return rng.uniform(lo, hi, n)


def test_two_prod_two_sum_are_exact():
    rng = np.random.default_rng(1)
    a = _rand(rng, 2000) * 10.0 ** rng.integers(-30, 30, 2000)
    b = _rand(rng, 2000) * 10.0 ** rng.integers(-30, 30, 2000)
    p, e = steps.two_prod(a, b)
    for i in range(2000):
        assert Fr(p[i]) + Fr(e[i]) == Fr(a[i]) * Fr(b[i])
    s, e = steps.two_sum(a, b)
    for i in range(2000):
        assert Fr(s[i]) + Fr(e[i]) == Fr(a[i]) + Fr(b[i])
        assert s[i] == a[i] + b[i]


def _unit_rows(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_accu_dop_bound_and_literal_variant_fails():
    """Sec. 5.2: |(dop+err) - (ad-bc)| / |ad-bc| <= (1 + 2(|ad|+|bc|)/|ad-bc|) u^2 + O(u^3)."""
    rng = np.random.default_rng(2)
    x1 = _unit_rows(rng, 3000)
    # nearly parallel partners make ad - bc cancel heavily
    x2 = x1 + rng.standard_normal((3000, 3)) * 10.0 ** rng.uniform(-12, 0, (3000, 1))
    x2 /= np.linalg.norm(x2, axis=1, keepdims=True)
    abcd = np.stack([x1[:, 1], x1[:, 2], x2[:, 1], x2[:, 2]], axis=1)  # y1 z2 - z1 y2
    worst = {0: 0.0, steps.LITERAL_DOP: 0.0}
    for var in worst:
        dop, err = steps.accu_dop(abcd, variant=var)
        for i in range(3000):
            a, b, c, d = (Fr(v) for v in abcd[i])
            ex = a * d - b * c
            if ex == 0:
                continue
            bound = (1 + 2 * (abs(a * d) + abs(b * c)) / abs(ex)) * Uf * Uf
            ratio = abs(Fr(dop[i]) + Fr(err[i]) - ex) / abs(ex) / bound
            worst[var] = max(worst[var], float(ratio))
    assert worst[0] <= 1.0 + 1e-6
    assert worst[steps.LITERAL_DOP] > 1e6


def test_renormalised_accu_dop_is_same_value():
    """Reading R8: one TwoSum after AccuDOP changes the pair, not its sum."""
    rng = np.random.default_rng(3)
    abcd = rng.uniform(-1, 1, (1000, 4))
    d0, e0 = steps.accu_dop(abcd, variant=0)
    d2, e2 = steps.accu_dop(abcd, variant=2)
    for i in range(1000):
        assert Fr(d0[i]) + Fr(e0[i]) == Fr(d2[i]) + Fr(e2[i])
        assert abs(e2[i]) <= U * abs(d2[i])


def test_comp_dot_c_bound():
    """Sec. 5.1: relative error <= gamma_n n u / (1 - (n-1) u) |x||y| / |x.y|."""
    rng = np.random.default_rng(4)
    for L in (2, 4, 6):
        x = rng.standard_normal((800, L))
        y = rng.standard_normal((800, L))
        # make about half the cases ill-conditioned
        y[:400, -1] = -(x[:400, :-1] * y[:400, :-1]).sum(1) / x[:400, -1]
        p, s = steps.comp_dot_c(x, y)
        g = L * Uf / (1 - L * Uf)
        for i in range(800):
            ex = sum(Fr(a) * Fr(b) for a, b in zip(x[i], y[i]))
            if ex == 0:
                continue
            absdot = sum(abs(Fr(a) * Fr(b)) for a, b in zip(x[i], y[i]))
            bound = g * L * Uf / (1 - (L - 1) * Uf) * absdot / abs(ex)
            assert abs(Fr(p[i]) + Fr(s[i]) - ex) / abs(ex) <= bound


def test_sum_non_neg_bound():
    """Algorithm 6: relative error <= 3 u^2 for non-negative pairs (Sec. 5.3)."""
    rng = np.random.default_rng(5)
    A = rng.uniform(0, 1, 2000) * 10.0 ** rng.integers(-8, 1, 2000)
    B = rng.uniform(0, 1, 2000) * 10.0 ** rng.integers(-8, 1, 2000)
    a, _ = steps.two_prod(A, rng.uniform(0, 1, 2000))
    pa = np.stack([A, A * U * rng.uniform(0, 1, 2000), B, B * U * rng.uniform(0, 1, 2000)], 1)
    S, s = steps.sum_non_neg(pa)
    for i in range(2000):
        ex = sum(Fr(v) for v in pa[i])
        assert abs(Fr(S[i]) + Fr(s[i]) - ex) <= 3 * Uf * Uf * ex


def test_sum_of_squares_c_bounds():
    """Supplement S2: for |n| <= 1 the 3D pair lies within
    |n|^2 +- 3u^2 (3|n|^2 + 4|n|_1 + 4) of the exact squared norm of x + e."""
    rng = np.random.default_rng(6)
    x = _unit_rows(rng, 1500) * rng.uniform(0.01, 1, (1500, 1))
    e = x * U * rng.uniform(-1, 1, (1500, 3))
    S, s = steps.sum_of_squares_c(x, e)
    for i in range(1500):
        v = [Fr(a) + Fr(b) for a, b in zip(x[i], e[i])]
        n2 = sum(t * t for t in v)
        n1 = sum(abs(t) for t in v)
        assert abs(Fr(S[i]) + Fr(s[i]) - n2) <= 3 * Uf * Uf * (3 * n2 + 4 * n1 + 4)
        assert abs(s[i]) <= U * abs(S[i])  # the closing FastTwoSum (Algorithm 7)


def test_acc_sqrt_bound():
    """AccSqrt (read as the Dekker/Taylor double-word square root): relative
    error of the pair <= 25/8 u^2 (Sec. 6.1, citing Rump 2023)."""
    rng = np.random.default_rng(7)
    S = rng.uniform(0, 1, 3000) * 10.0 ** rng.integers(-40, 2, 3000)
    e = S * U * rng.uniform(-1, 1, 3000)
    r, er = steps.acc_sqrt(S, e)
    from decimal import Decimal, getcontext
    getcontext().prec = 90
    worst = 0.0
    for i in range(3000):
        val = Fr(S[i]) + Fr(e[i])
        d = Decimal(val.numerator) / Decimal(val.denominator)
        ex = Fr(d.sqrt())
        rel = abs(Fr(r[i]) + Fr(er[i]) - ex) / ex
        worst = max(worst, float(rel / (Uf * Uf)))
    assert worst <= 25 / 8


def _norm_err(pts, ref, z0):
    rho = np.sqrt(np.maximum(0.0, (1 - z0) * (1 + z0)))
    d = pts - ref
    with np.errstate(invalid="ignore", divide="ignore"):
        e = np.sqrt(d[..., 0] ** 2 + d[..., 1] ** 2) / (U * rho[:, None])
    return np.nan_to_num(e)


def test_accux_meets_paper_bound_regime_ii():
    """Sec. 6.2: |P~ - P| <= 3 sqrt(1 - z0^2) u + h.o.t. away from tangency,
    for Algorithm 8 as printed and for the renormalised reading."""
    A, B, z = W.uniform_arcs(3000, seed=21)
    cnt, pts, fl = exact.intersect_batch(A, B, z)
    for var in (0, 2):
        c, p = steps.accux(A, B, z, variant=var)
        ok = fl == 0
        assert np.array_equal(c[ok], cnt[ok])
        assert _norm_err(p, pts, z)[ok].max() <= 3.0


def test_accux_renormalised_on_stress_mix():
    """Short, near-tangent, near-pole and near-antipodal arcs: the renormalised
    AccuX stays within the paper's bound; the printed one does not on short and
    near-antipodal arcs (the dropped e^2 terms of SumOfSquaresC)."""
    A, B, z, k = W.stress_arcs(4000, seed=22, return_class=True)
    cnt, pts, fl = exact.intersect_batch(A, B, z)
    ok = fl == 0
    c2, p2 = steps.accux(A, B, z, variant=2)
    assert np.array_equal(c2[ok], cnt[ok])
    e2 = _norm_err(p2, pts, z)[ok]
    assert e2.max() <= 3.0
    c0, p0 = steps.accux(A, B, z, variant=0)
    e0 = _norm_err(p0, pts, z)
    assert e0[(k == 3) & ok].max() > 1e3


def test_direct_obeys_section4_bound():
    """Sec. 4: |P~ - P| <= (21/s + 19 sqrt(2)/|n_xy|) u + h.o.t. for the direct
    evaluation; it loses about half the digits near tangency."""
    A, B, z = W.uniform_arcs(3000, seed=23)
    cnt, pts, fl = exact.intersect_batch(A, B, z)
    c, p = steps.direct(A, B, z)
    n = np.cross(A, B)
    nxy = np.hypot(n[:, 0], n[:, 1])
    nn = np.linalg.norm(n, axis=1)
    # s and |n_xy| of the non-unit normal n = x1 x x2, as in Eq. 2.2
    s = np.sqrt(np.maximum(nxy ** 2 - (nn * z) ** 2, 0))
    bound = 21 / np.maximum(s, 1e-300) + 19 * np.sqrt(2) / nxy
    d = p - pts
    err = np.nan_to_num(np.sqrt(d[..., 0] ** 2 + d[..., 1] ** 2) / U)
    ok = (fl == 0) & (c == cnt)
    assert (err[ok] <= 1.5 * bound[ok][:, None]).all()
    assert err[ok].max() > 10  # and it is visibly worse than AccuX


# ---- App. A: intermediate errors; the reflection assumption of Sec. 3 --------
def test_exact_intermediates_give_the_pinned_point():
    """-X / |n_xy|^2 from oracle.exact.intermediates rounds to the oracle's
    (independently rounded, pinned) slot-0 candidate."""
    A, B, z = W.uniform_arcs(300, seed=301)
    for i in range(300):
        it = exact.intermediates(A[i], B[i], z[i])
        ex = exact.setup(tuple(A[i]), tuple(B[i]), float(z[i]))
        if it["s"] is None or ex.S2i == 0:
            continue
        px = exact.candidate_point(ex, 1)[0]
        val = -it["X"] / it["S2"]
        assert abs(float(val) - px) <= 2.0 ** -52 * max(abs(px), 2.0 ** -60)


def test_app_a_intermediates_below_u_until_the_final_roundings():
    """App. A: averaged over the primary-dataset stand-in, every pair that
    Algorithm 8 carries (n, |n_xy|^2, |n|^2, s^2, s, the numerator) has a
    relative error below u; only the final single-double roundings reach ~u."""
    A, B, z = W.uniform_arcs(600, seed=302)
    mid = steps.accux_intermediates(A, B, z, variant=2)
    errs = {k: [] for k in ("n", "S2", "S3", "Q", "s", "X", "fl_S2", "fl_X")}
    for i in range(600):
        it = exact.intermediates(A[i], B[i], z[i])
        if it["s"] is None or it["Q"] == 0 or it["X"] == 0:
            continue

        def rel(pair_hi, pair_lo, ref):
            return abs(float((Fr(pair_hi) + Fr(pair_lo) - ref) / ref))
        for k in range(3):
            if it["n"][k] != 0:
                errs["n"].append(rel(mid["n"][i, k], mid["en"][i, k], it["n"][k]))
        errs["S2"].append(rel(mid["S2"][i], mid["s2"][i], it["S2"]))
        errs["S3"].append(rel(mid["S3"][i], mid["s3"][i], it["S3"]))
        errs["Q"].append(rel(mid["ss2"][i], mid["ess2"][i], it["Q"]))
        errs["s"].append(rel(mid["sb"][i], mid["es"][i], it["s"]))
        errs["X"].append(rel(mid["X"][i], 0.0, it["X"]))
        errs["fl_S2"].append(rel(mid["S2"][i], 0.0, it["S2"]))
        errs["fl_X"].append(rel(mid["X"][i], 0.0, it["X"]))
    mean = {k: float(np.mean(v)) for k, v in errs.items()}
    for k in ("n", "S2", "S3", "Q", "s"):
        assert mean[k] < 2.0 ** -80, (k, mean[k])   # pairs: O(u^2), far below u
    for k in ("X", "fl_S2", "fl_X"):
        assert mean[k] < U, (k, mean[k])             # single doubles: below u on average


def _reflect(A, B, z, axis):
    A2, B2, z2 = A.copy(), B.copy(), z.copy()
    A2[:, axis] = -A2[:, axis]
    B2[:, axis] = -B2[:, axis]
    if axis == 2:
        z2 = -z2
    return A2, B2, z2


def expected_after(pts, axis):
    """Points of the original arcs mapped by a reflection (axis 0, 1, 2) or an
    endpoint swap ('swap'): coordinate signs and, where the sign of the s-term
    of Eq. 2.2 flips (z reflection, swap), the two slots exchanged."""
    out = pts.copy()
    if axis in (0, 1):
        out[..., axis] = -out[..., axis]
        return out
    out = out[:, ::-1, :].copy()
    if axis == 2:
        out[..., 2] = -out[..., 2]
    return out


def equal_as_mapped(c, got, want):
    """Bitwise equality of mapped outputs: two-hit arcs slot by slot, one-hit
    arcs by their point (a tangent point is always reported in slot 0, so a
    slot-exchanging map leaves it there), no-hit arcs all NaN."""
    got = np.asarray(got)
    want = np.asarray(want)
    two = c == 2
    if not np.array_equal(got[two].view(np.int64), want[two].view(np.int64)):
        return False
    for i in np.flatnonzero(c == 1):
        g = got[i][np.isfinite(got[i, :, 0])]
        w = want[i][np.isfinite(want[i, :, 0])]
        if g.shape != (1, 3) or not np.array_equal(g.view(np.int64), w.view(np.int64)):
            return False
    return bool(np.isnan(got[c <= 0]).all() and np.isnan(want[c <= 0]).all())


@pytest.mark.parametrize("axis", [0, 1, 2, "swap"])
def test_step_reference_is_reflection_equivariant(axis):
    """Sec. 3 reduces the analysis to n >= 0, z0 >= 0 by reflections, as if
    nothing were lost by doing so. In round-to-nearest arithmetic every step of
    Algorithm 8 (and of the direct form) commutes with negations and
    operand swaps, so the reduction holds bit for bit."""
    A, B, z = W.stress_arcs(4000, seed=303)
    for fn in (lambda a, b, c: steps.accux(a, b, c, variant=2), steps.direct):
        c0, p0 = fn(A, B, z)
        if axis == "swap":
            c1, p1 = fn(B, A, z)
        else:
            c1, p1 = fn(*_reflect(A, B, z, axis))
        assert np.array_equal(c0, c1)
        assert equal_as_mapped(c0, p1, expected_after(p0, axis))
