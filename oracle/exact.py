"""Exact-rational oracle for one great circle arc against one constant latitude.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may use this module.

What it computes (the plain definition)
---------------------------------------
The inputs x1, x2 (FP64 3-vectors) and z0 (FP64) are taken as exact reals
(Sec. 3). With the exact normal n = x1 x x2 (Sec. 1.2), S2 = nx^2 + ny^2,
S3 = |n|^2 and Q = S2 - S3 z0^2, the candidate points are Eq. 2.2:

    P(sigma) = ( -(z0 nx nz + sigma s ny) / S2,
                 -(z0 ny nz - sigma s nx) / S2,
                  z0 ),        s = sqrt(Q),  sigma = +1 or -1.

sigma = +1 is the root the paper's AccuX returns (the alpha* <= 0 solution,
Sec. 2 and Algorithm 8); it is output slot 0, sigma = -1 is slot 1.
The circles meet iff Q >= 0, in two points iff Q > 0 (Sec. 2). A candidate is
a hit iff it lies on the closed minor arc from x1 to x2, which we decide as
(x1 x P) . n >= 0 and (P x x2) . n >= 0 (Sec. 2 only says the point must lie
"between" the endpoints; this is our reading). Each coordinate of a hit is the
exact value correctly rounded to nearest, ties to even (Sec. 3).

How
---
Every FP64 input is an integer times a power of two, so after scaling by a
common power of two, n, S2, S3 and Q are exact Python integers. A candidate is
then c * P = U + sigma * sqrt(Q) * V with integer vectors U, V and integer
c > 0, so every sign question is the sign of alpha + beta * sqrt(Q) with
integers alpha, beta, decided exactly, and every coordinate is
(alpha + beta * sqrt(Q)) / c, rounded by bracketing sqrt(Q) with integer
square roots at growing precision until both bracket ends round alike
(a Ziv loop; the value is irrational unless Q is a perfect square, in which
case it is rounded exactly as a rational).

Conventions shared with the C-ABI (our readings, where the paper is silent)
--------------------------------------------------------------------------
count = -1 : degenerate arc (n = 0), or the arc's great circle is the equator
             and z0 = 0 (coincident circles).
count = 0  : no hit; also for non-finite inputs.
Q == 0     : tangency, one candidate, reported in slot 0.
Unused slots hold NaN (all three coordinates).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction

# near-boundary flag bits (cases where a floating-point decision may
# legitimately differ from the exact one; see flags_of())
FLAG_NEAR_TANGENT = 1   # |Q| <= 2^-96 * S2: sign of s^2 ill-conditioned
FLAG_NEAR_ENDPOINT = 2  # a candidate lies within angle 2^-40 of x1 or x2
FLAG_TINY_NORMAL = 4    # |n| < 2^-200 |x1||x2|: arc shorter than ~1e-60 rad
FLAG_NONFINITE = 8      # an input is NaN or infinite

TANGENT_LOG2 = 96
ENDPOINT_LOG2 = 40
TINY_NORMAL_LOG2 = 200

_NAN = float("nan")


# ----------------------------------------------------------------- rounding --
def round_rational(num: int, den: int) -> float:
    """num/den correctly rounded to the nearest binary64, ties to even.

    Handles subnormal results (exponent floor 2^-1074) and returns +-inf when
    the rounded magnitude exceeds the largest finite double (IEEE 754
    round-to-nearest overflow rule, Sec. 3).
    """
    if den <= 0:
        raise ValueError("den must be positive")
    if num == 0:
        return 0.0
    neg = num < 0
    num = -num if neg else num
    # choose e so that the integer quotient q = floor(num / (den * 2^e)) has
    # exactly 53 bits, unless that would put e below the subnormal floor
    e = num.bit_length() - den.bit_length() - 53
    while True:
        if e < -1074:
            e = -1074
        if e >= 0:
            d = den << e
            q, r = divmod(num, d)
        else:
            d = den
            q, r = divmod(num << (-e), den)
        if q >= (1 << 53):
            e += 1
            continue
        if q < (1 << 52) and e > -1074:
            e -= 1
            continue
        break
    # round half to even on the remainder r / d
    twice = 2 * r
    if twice > d or (twice == d and (q & 1)):
        q += 1
    if q == (1 << 53):
        q >>= 1
        e += 1
    if e + 53 > 1024:  # q * 2^e >= 2^1024
        val = math.inf
    else:
        val = math.ldexp(q, e)
    return -val if neg else val


def round_quadratic(alpha: int, beta: int, Q: int, c: int) -> float:
    """(alpha + beta*sqrt(Q)) / c correctly rounded to binary64 (c > 0, Q >= 0)."""
    if Q < 0 or c <= 0:
        raise ValueError("need Q >= 0 and c > 0")
    if beta == 0 or Q == 0:
        return round_rational(alpha, c)
    r = math.isqrt(Q)
    if r * r == Q:  # sqrt(Q) is an integer: the value is rational
        return round_rational(alpha + beta * r, c)
    k = 64
    while True:
        r = math.isqrt(Q << (2 * k))  # r < sqrt(Q) * 2^k < r + 1 (irrational)
        lo = alpha * (1 << k) + beta * r
        hi = lo + beta
        a = round_rational(lo, c << k)
        b = round_rational(hi, c << k)
        if a == b:
            return a
        k *= 2


def sign_quadratic(alpha: int, beta: int, Q: int) -> int:
    """Exact sign of alpha + beta*sqrt(Q) for integers, Q >= 0."""
    if Q < 0:
        raise ValueError("Q must be >= 0")
    sa = (alpha > 0) - (alpha < 0)
    sb = (beta > 0) - (beta < 0)
    if Q == 0 or sb == 0:
        return sa
    if sa == 0 or sa == sb:
        return sb
    # opposite signs: compare alpha^2 with beta^2 * Q
    lhs = alpha * alpha
    rhs = beta * beta * Q
    if lhs > rhs:
        return sa
    if lhs < rhs:
        return sb
    return 0


# ------------------------------------------------------------ exact setup --
def dyadic(x: float) -> tuple[int, int]:
    """x = m * 2^e exactly, with integer m (m odd or zero)."""
    num, den = float(x).as_integer_ratio()
    if num == 0:
        return 0, 0
    e = -(den.bit_length() - 1)
    while num % 2 == 0:
        num //= 2
        e += 1
    return num, e


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1],
            a[2] * b[0] - a[0] * b[2],
            a[0] * b[1] - a[1] * b[0])


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


@dataclass
class ExactArc:
    """Exact integer data of one arc/latitude pair (all quantities scaled).

    x1 = X1 * 2^E, x2 = X2 * 2^E, z0 = Z / 2^F, n = N * 2^(2E),
    S2 = S2i * 2^(4E), S3 = S3i * 2^(4E), Q = Qi * 2^(4E - 2F),
    candidate(sigma) = (U + sigma * sqrt(Qi) * V) / c with c = S2i * 2^F.
    """
    X1: tuple
    X2: tuple
    E: int
    Z: int
    F: int
    N: tuple
    S2i: int
    S3i: int
    Qi: int
    c: int
    U: tuple
    V: tuple


def setup(x1, x2, z0) -> ExactArc:
    """Scale the FP64 inputs to integers and form n, S2, S3, Q exactly (Eq. 2.2)."""
    parts = [dyadic(v) for v in (*x1, *x2)]
    exps = [e for m, e in parts if m != 0]
    E = min(exps) if exps else 0
    ints = [m << (e - E) if m != 0 else 0 for m, e in parts]
    X1, X2 = tuple(ints[:3]), tuple(ints[3:])
    zm, ze = dyadic(z0)
    if ze >= 0:
        Z, F = zm << ze, 0
    else:
        Z, F = zm, -ze
    N = _cross(X1, X2)
    S2i = N[0] * N[0] + N[1] * N[1]
    S3i = S2i + N[2] * N[2]
    Qi = (S2i << (2 * F)) - S3i * Z * Z
    c = S2i << F
    U = (-Z * N[0] * N[2], -Z * N[1] * N[2], Z * S2i)
    V = (-N[1], N[0], 0)
    return ExactArc(X1, X2, E, Z, F, N, S2i, S3i, Qi, c, U, V)


def contained_sign(ex: ExactArc, sigma: int) -> tuple[int, int]:
    """Exact signs of t1 = (x1 x P).n and t2 = (P x x2).n for candidate sigma.

    Positive scale factors are dropped; t = alpha + sigma*beta*sqrt(Qi).
    """
    Q = max(ex.Qi, 0)
    a1 = _dot(_cross(ex.X1, ex.U), ex.N)
    b1 = _dot(_cross(ex.X1, ex.V), ex.N)
    a2 = _dot(_cross(ex.U, ex.X2), ex.N)
    b2 = _dot(_cross(ex.V, ex.X2), ex.N)
    return (sign_quadratic(a1, sigma * b1, Q), sign_quadratic(a2, sigma * b2, Q))


def _approx_sine(alpha: int, beta: int, Q: int, scale: Fraction) -> float:
    """|alpha + beta*sqrt(Q)| * scale as a float, accurate enough for a flag."""
    k = 80
    r = math.isqrt(Q << (2 * k))  # sqrt(Q) to within 2^-80
    val = abs(Fraction((alpha << k) + beta * r, 1 << k))
    return float(val * scale)


def _norm_int(v) -> int:
    return max(math.isqrt(_dot(v, v)), 1)


def flags_of(ex: ExactArc, candidates) -> int:
    """Near-boundary flags: where a correct floating-point kernel may differ.

    FLAG_NEAR_TANGENT when |Q| <= 2^-96 S2 (the computed sign of s^2 is only
    reliable above an O(u^2) error, Sec. 6.1); FLAG_NEAR_ENDPOINT when a
    candidate is within angle 2^-40 of an endpoint (containment near a tie);
    FLAG_TINY_NORMAL for arcs so short that |n| is below 2^-200 |x1||x2|.
    """
    fl = 0
    n2 = _dot(ex.N, ex.N)
    if (n2 << (2 * TINY_NORMAL_LOG2)) < _dot(ex.X1, ex.X1) * _dot(ex.X2, ex.X2):
        fl |= FLAG_TINY_NORMAL
    if ex.S2i > 0 and (abs(ex.Qi) << TANGENT_LOG2) <= (ex.S2i << (2 * ex.F)):
        fl |= FLAG_NEAR_TANGENT
    if ex.Qi >= 0 and ex.S2i > 0:
        Q = ex.Qi
        nN = _norm_int(ex.N)
        for sigma in candidates:
            a1 = _dot(_cross(ex.X1, ex.U), ex.N)
            b1 = sigma * _dot(_cross(ex.X1, ex.V), ex.N)
            a2 = _dot(_cross(ex.U, ex.X2), ex.N)
            b2 = sigma * _dot(_cross(ex.V, ex.X2), ex.N)
            # |c P| = c exactly because P is a unit vector
            s1 = _approx_sine(a1, b1, Q, Fraction(1, _norm_int(ex.X1) * ex.c * nN))
            s2 = _approx_sine(a2, b2, Q, Fraction(1, _norm_int(ex.X2) * ex.c * nN))
            if min(s1, s2) < 2.0 ** -ENDPOINT_LOG2:
                fl |= FLAG_NEAR_ENDPOINT
    return fl


def candidate_point(ex: ExactArc, sigma: int) -> tuple[float, float, float]:
    """Correctly rounded coordinates of candidate sigma (requires Qi >= 0, S2i > 0)."""
    Q = ex.Qi
    px = round_quadratic(ex.U[0], sigma * ex.V[0], Q, ex.c)
    py = round_quadratic(ex.U[1], sigma * ex.V[1], Q, ex.c)
    pz = round_rational(ex.Z, 1 << ex.F)
    return (px, py, pz)


@dataclass
class Result:
    count: int
    pts: list = field(default_factory=lambda: [[_NAN] * 3, [_NAN] * 3])
    flags: int = 0


def intersect(x1, x2, z0) -> Result:
    """Exact hits of the minor arc x1->x2 with the latitude z = z0 (Sec. 1.2, Eq. 2.2)."""
    vals = (*x1, *x2, z0)
    if not all(math.isfinite(float(v)) for v in vals):
        return Result(0, flags=FLAG_NONFINITE)
    ex = setup(tuple(float(v) for v in x1), tuple(float(v) for v in x2), float(z0))
    if ex.N == (0, 0, 0):
        return Result(-1, flags=flags_of(ex, ()))
    if ex.S2i == 0:
        # the great circle is the equator: coincident if z0 = 0, else disjoint
        return Result(-1 if ex.Z == 0 else 0, flags=flags_of(ex, ()))
    if ex.Qi < 0:
        return Result(0, flags=flags_of(ex, ()))
    sigmas = (1,) if ex.Qi == 0 else (1, -1)
    res = Result(0)
    for slot, sigma in enumerate(sigmas):
        g1, g2 = contained_sign(ex, sigma)
        if g1 >= 0 and g2 >= 0:
            res.pts[slot] = list(candidate_point(ex, sigma))
            res.count += 1
    res.flags = flags_of(ex, sigmas)
    return res


# ---------------------------------------------------------------- batches --
def _batch_worker(args):
    A, B, Z = args
    out = []
    for i in range(len(Z)):
        r = intersect(A[i], B[i], Z[i])
        out.append((r.count, r.pts, r.flags))
    return out


def intersect_batch(A, B, z0, processes: int | None = None):
    """Run intersect() over arrays A (n,3), B (n,3), z0 (n,).

    Returns (count int32[n], pts float64[n,2,3], flags int32[n]).
    processes > 1 uses a 'spawn' process pool (safe after CUDA has started).
    """
    import numpy as np
    A = np.asarray(A, dtype=np.float64).reshape(-1, 3)
    B = np.asarray(B, dtype=np.float64).reshape(-1, 3)
    z0 = np.asarray(z0, dtype=np.float64).reshape(-1)
    n = z0.shape[0]
    count = np.zeros(n, dtype=np.int32)
    pts = np.full((n, 2, 3), np.nan)
    flags = np.zeros(n, dtype=np.int32)
    Al, Bl, Zl = A.tolist(), B.tolist(), z0.tolist()
    if processes is None or processes <= 1 or n < 2048:
        rows = _batch_worker((Al, Bl, Zl))
    else:
        import multiprocessing as mp
        chunk = (n + processes * 4 - 1) // (processes * 4)
        jobs = [(Al[i:i + chunk], Bl[i:i + chunk], Zl[i:i + chunk])
                for i in range(0, n, chunk)]
        with mp.get_context("spawn").Pool(processes) as pool:
            rows = [r for part in pool.map(_batch_worker, jobs) for r in part]
    for i, (c, p, f) in enumerate(rows):
        count[i] = c
        pts[i] = p
        flags[i] = f
    return count, pts, flags


# ------------------------------------------------------------ intermediates --
def intermediates(x1, x2, z0, bits: int = 256):
    """Exact values of the quantities Algorithm 8 carries (App. A), as Fractions:
    n (3 components), |n_xy|^2, |n|^2, s^2, s = sqrt(s^2) and the root-0
    numerator X = z0 n_x n_z + s n_y of the x-coordinate (P_x = -X / |n_xy|^2).
    s and X are irrational: they are given to within 2^-bits relative."""
    ex = setup(tuple(float(v) for v in x1), tuple(float(v) for v in x2), float(z0))
    n = [Fraction(v) * Fraction(2) ** (2 * ex.E) for v in ex.N]
    S2 = n[0] ** 2 + n[1] ** 2
    S3 = S2 + n[2] ** 2
    z = Fraction(float(z0))
    Q = S2 - S3 * z * z
    s = None
    if Q >= 0:
        num, den = Q.numerator, Q.denominator
        k = bits + max(0, den.bit_length() - num.bit_length())
        r = math.isqrt((num << (2 * k)) // den)  # sqrt(Q) 2^k, truncated
        s = Fraction(r, 1 << k)
    X = z * n[0] * n[2] + s * n[1] if s is not None else None
    return {"n": n, "S2": S2, "S3": S3, "Q": Q, "s": s, "X": X}
