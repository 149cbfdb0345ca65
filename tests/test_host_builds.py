"""The integer-limb arithmetic of the headline kernel, built for the host, against
exact rationals (no GPU).

The 96-bit routines the intersection formula relies on must meet the error
bounds the kernel's accuracy argument uses:
  * the reciprocal and the square root (FP32 seed, fixed-point Newton steps
    with residuals read from the products' middle limbs) within 2^-92 relative;
  * products (top limbs kept) and sums (truncating alignment) within a few
    units of 2^-96 relative to their operands;
  * the conversion to FP64 rounds to nearest, ties to even, exactly.
Seeded random mantissas plus the edge cases of each routine: f = 1/2, f just
below 1, mantissas next to the FP32 seed's rounding steps, odd and even
exponents, cancellation in sums.

The kernels' per-pair evaluations are built for the host too (nvcc, host code
only, no FMA contraction) and checked on the CPU:
  * integer limbs (latitude and arc x arc): the exact oracle's hit counts on
    unflagged arcs and its correctly rounded points, bit for bit;
  * float-float: its stated bound;
  * AccuX (renormalised and as printed) and direct FP64: the step-by-step FP64
    reference, bit for bit;
  * the adaptive filter's error bound: every arc it keeps has the exact hit
    count (near-boundary arcs included) and points within the gate;
  * the band-area routines (boundary integral, fan, fan plus sliver): the
    band-area oracle within 32 u (longitude perimeter + height range);
  * the height range of each arc that decides its candidate latitudes: it
    contains the arc's exact height extent (so no hit is lost) and is widened
    by no more than the FP32 margin;
  * the latitude searches, against numpy.searchsorted;
  * the zonal sums' 128-bit fixed point: each term rounded once to a multiple
    of 2^-80 (halves away from zero), and a sum back to the nearest double.
"""
import ctypes
import os
import random
import shutil
import subprocess
from fractions import Fraction as F

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host_build_limbs.cpp")
OUT = os.path.join(ROOT, "paper_2510_09892_gb300", "_build", "host_build_limbs.so")
PAIR_SRC = os.path.join(ROOT, "tests", "host_build_kernels.cu")
PAIR_OUT = os.path.join(ROOT, "paper_2510_09892_gb300", "_build", "host_build_kernels.so")
TOP = 1 << 95


@pytest.fixture(scope="module")
def lib():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-o", OUT, SRC], check=True)
    L = ctypes.CDLL(OUT)
    u3 = ctypes.POINTER(ctypes.c_uint32)
    ip = ctypes.POINTER(ctypes.c_int)
    L.h_recip.argtypes = [u3, ctypes.c_int, ctypes.c_int, u3, ip, ip]
    L.h_sqrt.argtypes = [u3, ctypes.c_int, u3, ip, ip]
    for f in (L.h_mul, L.h_add):
        f.argtypes = [u3, ctypes.c_int, ctypes.c_int, u3, ctypes.c_int, ctypes.c_int, u3, ip, ip]
    L.h_to_double.argtypes = [u3, ctypes.c_int, ctypes.c_int]
    L.h_to_double.restype = ctypes.c_double
    L.h_check_seeds.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint32)]
    L.h_check_seeds.restype = ctypes.c_uint64
    return L


@pytest.mark.parametrize("which", ["rcp32", "rsqrt32"])
def test_host_fp32_seeds_are_correctly_rounded(lib, which):
    """The FP32 seeds of the integer-limb reciprocal and square root: the
    host forms (through FP64) equal the correctly rounded value on every float
    of one binade (two for the square root), so they equal the device's
    correctly rounded __frcp_rn / __frsqrt_rn bit for bit. (The on-arc test's
    normalisation factor, rsqrt_approx, is rsqrtf on the device and
    1 / sqrtf on the host: that one factor may differ in its last bits, which
    moves no decision outside the oracle's near-endpoint flag, so the host
    builds are checked against the oracle there, not against the device.)"""
    bad = ctypes.c_uint32()
    n = lib.h_check_seeds(0 if which == "rcp32" else 1, ctypes.byref(bad))
    assert n == 0, (n, hex(bad.value))


def limbs(M):
    return (ctypes.c_uint32 * 3)(M & 0xffffffff, (M >> 32) & 0xffffffff, M >> 64)


def value(M, e, neg=0):
    v = F(M, 1 << 96) * F(2) ** e
    return -v if neg else v


def call(fn, *args):
    r = (ctypes.c_uint32 * 3)()
    e, n = ctypes.c_int(), ctypes.c_int()
    fn(*args, r, ctypes.byref(e), ctypes.byref(n))
    R = r[0] | (r[1] << 32) | (r[2] << 64)
    return R, e.value, n.value


def mantissas(rng, n):
    out = [TOP, TOP + 1, (1 << 96) - 1, (1 << 96) - 2, TOP | (1 << 72), TOP + (1 << 71)]
    for _ in range(200):  # next to the 24-bit seed's rounding steps
        t = rng.randrange(1 << 23, 1 << 24)
        out.append(min((1 << 96) - 1, max(TOP, (t << 72) + rng.randrange(-(1 << 66), 1 << 66))))
    out += [rng.randrange(TOP, 1 << 96) for _ in range(n)]
    return out


def rel(got, exact):
    return abs((got - exact) / exact)


def test_reciprocal_within_2_pow_minus_92(lib):
    rng = random.Random(20251009)
    worst = 0
    for M in mantissas(rng, 3000):
        for e, neg in ((0, 0), (1, 1), (-37, 0), (600, 1)):
            R, er, nr = call(lib.h_recip, limbs(M), e, neg)
            assert R >> 95 == 1 and nr == neg
            worst = max(worst, rel(value(R, er, nr), 1 / value(M, e, neg)))
    assert worst <= F(1, 1 << 92), float(worst)
    # 1/2 and 2 are exact
    R, er, _ = call(lib.h_recip, limbs(TOP), 0, 0)
    assert value(R, er) == 2


def test_square_root_within_2_pow_minus_92(lib):
    import math
    rng = random.Random(20251010)
    worst = 0
    for M in mantissas(rng, 3000):
        for e in (0, 1, -5, 8, -1021):
            R, er, nr = call(lib.h_sqrt, limbs(M), e)
            assert R >> 95 == 1 and nr == 0
            a = value(M, e)
            got = value(R, er)
            # |got - sqrt(a)| = |got^2 - a| / (got + sqrt(a)), with sqrt(a) from an integer
            # square root of a 2^p (p even, large enough to leave 150 bits)
            t = e - 96
            p = max(300, 300 - t)
            p += p & 1
            s = F(math.isqrt(M << (t + p)), 1 << (p // 2))
            worst = max(worst, abs(got * got - a) / (got + s) / s)
    assert worst <= F(1, 1 << 92), float(worst)
    # perfect squares: 1/4 and its powers of four
    for e in (0, 2, -40):
        R, er, _ = call(lib.h_sqrt, limbs(TOP), e - 1)  # 2^(e - 2)
        assert abs(value(R, er) - F(2) ** ((e - 2) // 2)) <= F(2) ** ((e - 2) // 2) / (1 << 92)


def test_products_and_sums_within_a_few_units_of_2_pow_minus_96(lib):
    rng = random.Random(7)
    unit = F(1, 1 << 96)
    for _ in range(3000):
        A, B = rng.randrange(TOP, 1 << 96), rng.randrange(TOP, 1 << 96)
        ea, eb = rng.randrange(-40, 40), rng.randrange(-40, 40)
        na, nb = rng.randrange(2), rng.randrange(2)
        a, b = value(A, ea, na), value(B, eb, nb)
        R, er, nr = call(lib.h_mul, limbs(A), ea, na, limbs(B), eb, nb)
        assert rel(value(R, er, nr), a * b) <= 8 * unit
        R, er, nr = call(lib.h_add, limbs(A), ea, na, limbs(B), eb, nb)
        # truncating alignment: within a few units of the larger operand
        assert abs(value(R, er, nr) - (a + b)) <= 4 * unit * max(abs(a), abs(b))
    # exact cancellation gives zero; near cancellation is exact
    R, er, nr = call(lib.h_add, limbs(TOP + 5), 0, 0, limbs(TOP + 5), 0, 1)
    assert R == 0
    R, er, nr = call(lib.h_add, limbs(TOP + 5), 0, 0, limbs(TOP + 3), 0, 1)
    assert value(R, er, nr) == F(2, 1 << 96)


def test_conversion_to_double_rounds_to_nearest_even(lib):
    rng = random.Random(11)
    for _ in range(3000):
        M = rng.randrange(TOP, 1 << 96)
        if rng.random() < 0.3:  # exact ties and their neighbours
            M = (M >> 43 << 43) | (1 << 42) | rng.choice([0, 0, 1])
        e, neg = rng.randrange(-100, 100), rng.randrange(2)
        got = lib.h_to_double(limbs(M), e, neg)
        assert F(got) == F(float(value(M, e, neg)))  # Python rounds a Fraction to nearest even


@pytest.fixture(scope="module")
def pair_lib():
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc"
                                     if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("no nvcc for the host build of the pair evaluation")
    os.makedirs(os.path.dirname(PAIR_OUT), exist_ok=True)
    subprocess.run([nvcc, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC,-ffp-contract=off",
                    "-o", PAIR_OUT, PAIR_SRC], check=True)
    L = ctypes.CDLL(PAIR_OUT)
    L.h_pair_wide.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_longlong, ctypes.c_void_p,
                                                       ctypes.c_void_p]
    L.h_arcs_wide.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_longlong, ctypes.c_void_p,
                                                       ctypes.c_void_p]
    for f in (L.h_pair_ff32, L.h_pair_direct, L.h_pair_accux, L.h_pair_accux_printed):
        f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p]
    L.h_pair_filtered.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_longlong, ctypes.c_double,
                                                          ctypes.c_void_p, ctypes.c_void_p,
                                                          ctypes.c_void_p]
    vp, ll = ctypes.c_void_p, ctypes.c_longlong
    L.h_f32_of_mismatches.argtypes = [vp, ll]
    L.h_f32_of_mismatches.restype = ll
    L.h_green_cells.argtypes = [vp, ll, vp, vp, ll, vp, ll, vp, ctypes.c_int]
    L.h_green_cells.restype = ctypes.c_uint
    L.h_fan_cells.argtypes = [vp, ll, vp, vp, ll, vp, ctypes.c_int]
    L.h_pair_cells.argtypes = [vp, ll, vp, vp, ll, vp, ll, vp, vp, ctypes.c_int]
    L.h_z_ranges.argtypes = [vp, vp, ll, vp, vp, vp, vp]
    L.h_rcp_den.argtypes = [vp, ll, vp]
    L.h_unit.argtypes = [vp, ll, vp]
    L.h_compares.argtypes = [vp, ll, vp]
    L.h_two_sum.argtypes = [vp, vp, ll, vp, vp]
    L.h_searches.argtypes = [vp, ll, vp, ll, vp, vp, vp]
    L.h_to_fixed.argtypes = [vp, ll, vp, vp, vp]
    L.h_from_fixed.argtypes = [vp, vp, ll, vp]
    L.h_accux_mid.argtypes = [vp, vp, vp, ll, vp]
    return L


@pytest.mark.parametrize("gen", ["uniform", "stress", "scaled"])
def test_pair_evaluation_on_the_host_matches_exact_oracle(pair_lib, gen):
    import numpy as np
    from oracle import exact
    from paper_2510_09892_gb300 import workloads as W
    if gen == "uniform":
        A, B, z = W.uniform_arcs(2000, seed=91)
    else:
        A, B, z = W.stress_arcs(2000, seed=92)
        if gen == "scaled":
            rng = np.random.default_rng(93)
            A = A * (10.0 ** rng.uniform(-30, 30, len(z)))[:, None]
            B = B * (10.0 ** rng.uniform(-30, 30, len(z)))[:, None]
    A, B, z = (np.ascontiguousarray(v, dtype=np.float64) for v in (A, B, z))
    n = len(z)
    pts = np.empty((n, 2, 3))
    cnt = np.empty(n, dtype=np.int32)
    pair_lib.h_pair_wide(A.ctypes.data, B.ctypes.data, z.ctypes.data, n, pts.ctypes.data,
                         cnt.ctypes.data)
    ce, pe, fe = exact.intersect_batch(A, B, z, processes=1)
    ok = fe == 0
    assert ok.mean() > 0.9
    assert np.array_equal(cnt[ok], ce[ok])
    hit = np.isfinite(pe[..., 0]) & ok[:, None]
    assert np.array_equal(np.isfinite(pts[..., 0]) & ok[:, None], hit)
    # correctly rounded: the same doubles as the oracle on every unflagged hit
    assert np.array_equal(pts[hit][:, :2], pe[hit][:, :2])


@pytest.mark.parametrize("scaled", [False, True])
def test_arc_pairs_on_the_host_match_exact_oracle(pair_lib, scaled):
    """Arc x arc in integer limbs, the same source built for the host: the exact
    oracle's hit counts on unflagged pairs and its correctly rounded points."""
    import numpy as np
    from oracle import exact_arcs
    from paper_2510_09892_gb300 import workloads as W
    A1, A2, B1, B2 = W.arc_pairs(2000, seed=94)
    if scaled:
        sc = 10.0 ** np.random.default_rng(95).uniform(-30, 30, (4, len(A1), 1))
        A1, A2, B1, B2 = A1 * sc[0], A2 * sc[1], B1 * sc[2], B2 * sc[3]
    A1, A2, B1, B2 = (np.ascontiguousarray(v, dtype=np.float64) for v in (A1, A2, B1, B2))
    n = len(A1)
    pts = np.empty((n, 2, 3))
    cnt = np.empty(n, dtype=np.int32)
    pair_lib.h_arcs_wide(A1.ctypes.data, A2.ctypes.data, B1.ctypes.data, B2.ctypes.data, n,
                         pts.ctypes.data, cnt.ctypes.data)
    ce, pe, fe = exact_arcs.intersect_arcs_batch(A1, A2, B1, B2, processes=1)
    ok = fe == 0
    assert ok.mean() > 0.9
    assert np.array_equal(cnt[ok], ce[ok])
    hit = np.isfinite(pe[..., 0]) & ok[:, None]
    assert np.array_equal(np.isfinite(pts[..., 0]) & ok[:, None], hit)
    assert np.array_equal(pts[hit], pe[hit])


@pytest.mark.parametrize("gen", ["uniform", "stress", "mixed", "scaled", "near"])
def test_float_float_on_the_host_within_stated_bound(pair_lib, gen):
    """The float-float form, the same source built for the host: every unflagged
    hit within its stated bound |dP| <= 2^-44 sqrt(1 - z0^2), near tangency
    included (the cancelling steps are exact or 128-bit), and the exact
    oracle's hit counts on every unflagged arc."""
    import numpy as np
    from oracle import exact
    from paper_2510_09892_gb300 import workloads as W
    from tests import parity as P
    if gen == "uniform":
        A, B, z = W.uniform_arcs(3000, seed=96)
    elif gen == "stress":
        A, B, z = W.stress_arcs(3000, seed=97)
    elif gen == "mixed":
        A, B, z = W.mixed_chunk(9, size=3000)
    elif gen == "near":
        A, B, z = W.near_boundary_arcs(2000, seed=98)
    else:
        A, B, z = W.stress_arcs(3000, seed=99)
        sc = 10.0 ** np.random.default_rng(100).uniform(-30, 30, (2, len(z), 1))
        A, B = A * sc[0], B * sc[1]
    A, B, z = (np.ascontiguousarray(v, dtype=np.float64) for v in (A, B, z))
    n = len(z)
    pts = np.empty((n, 2, 3))
    cnt = np.empty(n, dtype=np.int32)
    pair_lib.h_pair_ff32(A.ctypes.data, B.ctypes.data, z.ctypes.data, n, pts.ctypes.data,
                         cnt.ctypes.data)
    ce, pe, fe = exact.intersect_batch(A, B, z, processes=1)
    ok = fe == 0
    assert np.array_equal(cnt[ok], ce[ok])
    hit = np.isfinite(pe[..., 0]) & ok[:, None]
    assert np.array_equal(np.isfinite(pts[..., 0]) & ok[:, None], hit)
    err = P.norm_error(pts, pe, z)
    assert np.nanmax(np.where(hit, err, 0)) <= P.FF_BOUND


def test_fast_fp32_conversion_equals_general_one(pair_lib):
    """f32_of (the range code's FP64 -> FP32 conversion) gives the bits of
    f32_scaled(x, 0) on every exponent (each of the 2048 exponent fields with
    random mantissas and both signs, zeros, subnormals, infinities, NaN)."""
    import numpy as np
    rng = np.random.default_rng(7)
    ex = np.repeat(np.arange(2048, dtype=np.uint64), 64)
    mant = rng.integers(0, 1 << 52, ex.size, dtype=np.uint64)
    sign = rng.integers(0, 2, ex.size, dtype=np.uint64)
    bits = (sign << np.uint64(63)) | (ex << np.uint64(52)) | mant
    x = np.ascontiguousarray(bits.view(np.float64))
    assert pair_lib.h_f32_of_mismatches(x.ctypes.data, x.size) == 0
    edge = np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** -126, 2.0 ** -127, 2.0 ** 127, 2.0 ** 128,
                     np.inf, -np.inf, np.nan, 5e-324, 1.9999999999999998])
    assert pair_lib.h_f32_of_mismatches(edge.ctypes.data, edge.size) == 0


@pytest.mark.parametrize("form", ["accux", "accux_printed", "direct"])
@pytest.mark.parametrize("gen", ["uniform", "stress", "axes"])
def test_fp64_forms_on_the_host_equal_step_reference(pair_lib, form, gen):
    """AccuX (renormalised and as printed) and direct FP64, the kernels' source
    built for the host, equal the step-by-step FP64 reference bit for bit: the
    same correctly rounded operations in the same order (TwoSum in its
    three-operation ordered form gives the same pairs). "axes" draws the
    endpoint coordinates and z0 from 0, -0, +-1/2, +-1 and random values, so
    that exact zeros, signed zeros and exact sums run through every step."""
    import numpy as np
    from oracle import steps
    from paper_2510_09892_gb300 import workloads as W
    from tests import parity as P
    if gen == "axes":
        rng = np.random.default_rng(112)
        vals = np.array([0.0, -0.0, 0.5, -0.5, 1.0, -1.0])
        A = np.where(rng.random((3000, 3)) < 0.6, rng.choice(vals, (3000, 3)),
                     rng.standard_normal((3000, 3)))
        B = np.where(rng.random((3000, 3)) < 0.6, rng.choice(vals, (3000, 3)),
                     rng.standard_normal((3000, 3)))
        z = np.where(rng.random(3000) < 0.5, rng.choice(vals, 3000), rng.uniform(-1, 1, 3000))
    else:
        A, B, z = (W.uniform_arcs(3000, seed=98) if gen == "uniform"
                   else W.stress_arcs(3000, seed=99))
    A, B, z = (np.ascontiguousarray(v, dtype=np.float64) for v in (A, B, z))
    n = len(z)
    pts = np.empty((n, 2, 3))
    cnt = np.empty(n, dtype=np.int32)
    fn = {"accux": pair_lib.h_pair_accux, "accux_printed": pair_lib.h_pair_accux_printed,
          "direct": pair_lib.h_pair_direct}[form]
    fn(A.ctypes.data, B.ctypes.data, z.ctypes.data, n, pts.ctypes.data, cnt.ctypes.data)
    if form == "direct":
        cr, pr = steps.direct(A, B, z)
    else:
        cr, pr = steps.accux(A, B, z, variant=2 if form == "accux" else 0)
    assert np.array_equal(cnt, cr)
    assert P.same_bits(pts, pr)


@pytest.mark.parametrize("gen,gate,min_kept", [("uniform", 4.0, 0.0), ("uniform", 64.0, 0.3),
                                               ("stress", 2.0 ** 20, 0.08),
                                               ("scaled", 2.0 ** 20, 0.0)])
def test_adaptive_filter_bound_on_the_host(pair_lib, gen, gate, min_kept):
    """The adaptive filter's running error bound, the kernel's source built for
    the host: every arc it keeps has the exact oracle's hit count (flagged arcs
    included) and points within the gate."""
    import numpy as np
    from oracle import exact
    from paper_2510_09892_gb300 import workloads as W
    from tests import parity as P
    if gen == "uniform":
        A, B, z = W.uniform_arcs(3000, seed=100)
    else:
        A, B, z = W.stress_arcs(3000, seed=101)
        if gen == "scaled":
            rng = np.random.default_rng(102)
            A = A * (10.0 ** rng.uniform(-30, 30, len(z)))[:, None]
            B = B * (10.0 ** rng.uniform(-30, 30, len(z)))[:, None]
    A, B, z = (np.ascontiguousarray(v, dtype=np.float64) for v in (A, B, z))
    n = len(z)
    pts = np.empty((n, 2, 3))
    cnt = np.empty(n, dtype=np.int32)
    kept = np.empty(n, dtype=np.int32)
    pair_lib.h_pair_filtered(A.ctypes.data, B.ctypes.data, z.ctypes.data, n, gate,
                             pts.ctypes.data, cnt.ctypes.data, kept.ctypes.data)
    k = kept == 1
    print(f"{gen}, gate {gate:g}: kept {k.mean():.3f}")
    assert k.mean() >= min_kept
    if not k.any():
        return
    ce, pe, fe = exact.intersect_batch(A[k], B[k], z[k], processes=1)
    assert np.array_equal(cnt[k], ce)
    hit = np.isfinite(pe[..., 0])
    assert np.array_equal(np.isfinite(pts[k][..., 0]), hit)
    _, _, g = P.component_errors(pts[k], pe, z[k])
    assert np.nanmax(np.where(hit[..., None], g, 0.0), initial=0.0) <= gate


def _area_tolerance(cells):
    """32 u (sum of |longitude steps| between nodes off the poles + height range)."""
    import numpy as np
    from oracle import areas as OA
    out = []
    for c in cells:
        v = np.asarray(c)
        zr = np.ptp(OA.breakpoints(c))
        v = v[np.hypot(v[:, 0], v[:, 1]) > 0]
        w = np.roll(v, -1, axis=0)
        d = np.arctan2(v[:, 0] * w[:, 1] - v[:, 1] * w[:, 0], v[:, 0] * w[:, 0] + v[:, 1] * w[:, 1])
        out.append(np.abs(d).sum() + zr)
    return 32.0 * 2.0 ** -53 * np.array(out)


@pytest.mark.parametrize("kind", ["polygons", "cubed_sphere"])
def test_band_area_routines_on_the_host_match_oracle(pair_lib, kind):
    """The boundary integral on every cell; the fan on the cells the oracle puts
    inside one interior band; the fan plus sliver on the cells it puts in two.
    Each routine gives the same bits whether it normalises the nodes itself or
    reads the normalised copy that sphx_band_areas makes once per node."""
    import numpy as np
    from oracle import areas as OA
    from paper_2510_09892_gb300 import workloads as W
    if kind == "polygons":
        nodes, off, fn = W.polygon_cells(48, seed=33, radius=(1e-3, 0.4))
        lat = W.latlon_latitudes(61)
    else:  # odd N: the poles lie inside cells; 30-degree bands, so that cells
        # of about 18 degrees lie in one or two of them
        nodes, off, fn = W.cubed_sphere_cells(5)
        lat = W.latlon_latitudes(7)
    nodes, off, fn, lat = (np.ascontiguousarray(v) for v in (nodes, off.astype(np.int64),
                                                              fn.astype(np.int32), lat))
    cells = W.cells_as_lists(nodes, off, fn)
    F, nb = len(off) - 1, len(lat) - 1
    ref = np.array(OA.band_areas_batch(cells, lat, processes=min(8, os.cpu_count() or 1)))
    tol = _area_tolerance(cells)
    args = (nodes.ctypes.data, len(nodes), off.ctypes.data, fn.ctypes.data, F)
    green = np.zeros((F, nb))
    st = pair_lib.h_green_cells(*args, lat.ctypes.data, len(lat), green.ctypes.data, 0)
    assert st == 0
    green_pre = np.zeros((F, nb))
    assert pair_lib.h_green_cells(*args, lat.ctypes.data, len(lat), green_pre.ctypes.data, 1) == 0
    assert np.array_equal(green, green_pre)
    assert (np.abs(green - ref) <= tol[:, None]).all(), (np.abs(green - ref) / tol[:, None]).max()
    # cells in one / two interior bands (by the oracle)
    inside = ref > tol[:, None]
    first = np.argmax(inside, axis=1)
    nbands = inside.sum(axis=1)
    interior = (first > 0) & (first + nbands < nb)
    one = np.flatnonzero((nbands == 1) & interior)
    next_band = inside[np.arange(F), np.minimum(first + 1, nb - 1)]
    two = np.flatnonzero((nbands == 2) & interior & next_band)
    fan = np.empty(F)
    pair_lib.h_fan_cells(*args, fan.ctypes.data, 0)
    fan_pre = np.empty(F)
    pair_lib.h_fan_cells(*args, fan_pre.ctypes.data, 1)
    assert np.array_equal(fan, fan_pre, equal_nan=True)
    done = one[np.isfinite(fan[one])]
    assert len(one) > 0 and len(done) >= 0.5 * len(one)
    assert (np.abs(fan[done] - ref[done].sum(axis=1)) <= tol[done]).all()
    lo = first.astype(np.int32)
    pr = np.empty(2 * F)
    pair_lib.h_pair_cells(*args, lat.ctypes.data, len(lat), lo.ctypes.data, pr.ctypes.data, 0)
    pr_pre = np.empty(2 * F)
    pair_lib.h_pair_cells(*args, lat.ctypes.data, len(lat), lo.ctypes.data, pr_pre.ctypes.data, 1)
    assert np.array_equal(pr, pr_pre, equal_nan=True)
    pr = pr.reshape(F, 2)
    done2 = two[np.isfinite(pr[two, 0])]
    assert len(two) > 0 and len(done2) >= 0.5 * len(two)
    want = np.stack([ref[done2, first[done2]], ref[done2, first[done2] + 1]], axis=1)
    assert (np.abs(pr[done2] - want) <= tol[done2, None]).all()
    print(f"{kind}: {F} cells, fan {len(done)}/{len(one)}, fan plus sliver {len(done2)}/{len(two)}")


@pytest.mark.parametrize("gen", ["uniform", "stress", "scaled", "cubed_sphere", "meshes"])
def test_candidate_height_ranges_contain_the_arcs(pair_lib, gen):
    import numpy as np
    from oracle import areas as OA
    from paper_2510_09892_gb300 import workloads as W
    if gen == "uniform":
        A, B, _ = W.uniform_arcs(3000, seed=103)
    elif gen in ("stress", "scaled"):
        A, B, _ = W.stress_arcs(3000, seed=104)
        if gen == "scaled":
            rng = np.random.default_rng(105)
            A = A * (10.0 ** rng.uniform(-30, 30, len(A)))[:, None]
            B = B * (10.0 ** rng.uniform(-30, 30, len(B)))[:, None]
    elif gen == "cubed_sphere":
        A, B = W.cubed_sphere_edges(16)
    else:
        b = W.ragged_meshes(4, 40, 400, seed=106, lat_min=180, lat_max=300)
        A, B = b["A"], b["B"]
    A, B = (np.ascontiguousarray(v, dtype=np.float64) for v in (A, B))
    n = len(A)
    zmin, zmax = np.empty(n), np.empty(n)
    ok = np.empty(n, dtype=np.int32)
    f32 = np.empty(n, dtype=np.int32)
    pair_lib.h_z_ranges(A.ctypes.data, B.ctypes.data, n, zmin.ctypes.data, zmax.ctypes.data,
                        ok.ctypes.data, f32.ctypes.data)
    assert ok.all()
    lo = np.empty(n)
    hi = np.empty(n)
    for i in range(n):
        zs = OA.breakpoints([tuple(A[i]), tuple(B[i])])
        lo[i], hi[i] = min(zs), max(zs)
    assert (zmin <= lo).all() and (zmax >= hi).all()
    assert ((zmax - zmin) - (hi - lo) <= 8 * 2.0 ** -19).all()


def test_fp32_height_range_refuses_non_finite_endpoints(pair_lib):
    """The candidate kernels test finiteness only before the FP64 height range:
    the FP32 range must give none for an endpoint with an infinite or NaN
    coordinate (any of the six, either sign, NaN payloads included) or one
    scaled to the largest doubles, while it gives one for the same arcs with
    finite unit endpoints."""
    import numpy as np
    from paper_2510_09892_gb300 import workloads as W
    A0, B0, _ = W.uniform_arcs(64, seed=108)
    bad_values = [np.inf, -np.inf, np.nan, -np.nan,
                  np.frombuffer(np.uint64(0x7ff0000000000001).tobytes(), np.float64)[0],
                  np.frombuffer(np.uint64(0xfff8dead00000000).tobytes(), np.float64)[0],
                  1.7e308, -1.7e308]
    rows_A, rows_B = [], []
    for v in bad_values:
        for k in range(6):
            A, B = A0.copy(), B0.copy()
            (A if k < 3 else B)[:, k % 3] = v
            rows_A.append(A)
            rows_B.append(B)
    A = np.ascontiguousarray(np.concatenate(rows_A + [A0]))
    B = np.ascontiguousarray(np.concatenate(rows_B + [B0]))
    n = len(A)
    zmin, zmax = np.empty(n), np.empty(n)
    ok = np.empty(n, dtype=np.int32)
    f32 = np.empty(n, dtype=np.int32)
    pair_lib.h_z_ranges(A.ctypes.data, B.ctypes.data, n, zmin.ctypes.data, zmax.ctypes.data,
                        ok.ctypes.data, f32.ctypes.data)
    bad = slice(0, n - len(A0))
    assert not f32[bad].any()
    finite = np.isfinite(A).all(1) & np.isfinite(B).all(1)
    assert not ok[bad][~finite[bad]].any()
    assert f32[n - len(A0):].all() and ok[n - len(A0):].all()


def test_fan_reciprocal_and_node_normalisation_on_the_host(pair_lib):
    """The area kernels' two FP64 shortcuts, against exact rationals (the
    reciprocal) and 200-bit arithmetic (the normalisation): the
    reciprocal of a fan triangle's denominator (FP32 seed, two Newton steps)
    within 1 ulp of 1/den over [1, 4] (random values, the ends, powers of two
    and their neighbours), and the normalisation of nodes whose squared norm is
    within 2^-20 of 1 (the series branch) as well as of others (the reciprocal
    square root), within 4 units of 2^-53 of the exact v / |v|, relative, per
    component."""
    import numpy as np
    from fractions import Fraction as Fr
    rng = np.random.default_rng(109)
    x = np.concatenate([rng.uniform(1.0, 4.0, 4000), [1.0, 2.0, 4.0, 3.0, 1.5],
                        np.nextafter([1.0, 2.0, 2.0, 4.0], [2.0, 1.0, 3.0, 3.0])])
    out = np.empty_like(x)
    pair_lib.h_rcp_den(x.ctypes.data, len(x), out.ctypes.data)
    err = np.array([abs(Fr(float(o)) - 1 / Fr(float(v))) / (1 / Fr(float(v))) for v, o in zip(x, out)],
                   dtype=float)
    assert err.max() <= 2.0 ** -52
    # nodes: unit to rounding, scaled by 1 + up to 2^-21 (series), and far from unit
    v = rng.standard_normal((3000, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    scale = np.concatenate([np.ones(1000), 1 + rng.uniform(-2.0 ** -22, 2.0 ** -22, 1000),
                            10.0 ** rng.uniform(-3, 3, 1000)])
    v = np.ascontiguousarray(v * scale[:, None])
    u = np.empty_like(v)
    pair_lib.h_unit(v.ctypes.data, len(v), u.ctypes.data)
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 200
    worst = 0.0
    for i in range(len(v)):
        r = 1 / mp.sqrt(sum(mp.mpf(float(c)) ** 2 for c in v[i]))
        for k in range(3):
            e = mp.mpf(float(v[i, k])) * r
            if e != 0:
                worst = max(worst, float(abs(mp.mpf(float(u[i, k])) - e) / abs(e)))
    assert worst <= 4 * 2.0 ** -53


def test_integer_comparisons_equal_the_fp64_ones(pair_lib):
    """The kernels test doubles on the integer pipe: x < 0.5, |x| <= 2^-9,
    x > 0, x >= 0, x <= 0, x == 0 and isfinite(x) must equal the FP64 tests for signed
    zeros, subnormals, the constants and their neighbours, infinities, NaNs of
    either sign and random doubles over the whole exponent range."""
    import numpy as np
    rng = np.random.default_rng(110)
    special = [0.0, -0.0, 5e-324, -5e-324, 0.5, -0.5, 2.0 ** -9, -(2.0 ** -9),
               np.inf, -np.inf, np.nan, -np.nan, 1.0, -1.0, 1e308, -1e308]
    special += list(np.nextafter([0.5, 0.5, 2.0 ** -9, 2.0 ** -9], [0, 1, 0, 1]))
    bits = rng.integers(0, 2 ** 63, 20000, dtype=np.uint64) | (
        rng.integers(0, 2, 20000, dtype=np.uint64) << np.uint64(63))
    x = np.ascontiguousarray(np.concatenate([np.array(special), bits.view(np.float64),
                                             rng.uniform(-1, 1, 5000)]))
    x[len(special) + 3] = np.frombuffer(np.uint64(0xfff8000000000001).tobytes(), np.float64)[0]
    out = np.empty(len(x), dtype=np.int32)
    pair_lib.h_compares(x.ctypes.data, len(x), out.ctypes.data)
    with np.errstate(invalid="ignore"):
        want = ((x < 0.5).astype(int) | ((np.abs(x) <= 2.0 ** -9).astype(int) << 1)
                | ((x > 0.0).astype(int) << 2) | ((x >= 0.0).astype(int) << 3)
                | ((x == 0.0).astype(int) << 4) | (np.isfinite(x).astype(int) << 5)
                | ((x <= 0.0).astype(int) << 6))
    assert np.array_equal(out, want)


def test_fp64_two_sum_equals_knuths_six_operations(pair_lib):
    """The kernels' FP64 TwoSum (operands ordered by magnitude on the integer
    pipe, then FastTwoSum) gives the pair of Knuth's six-operation TwoSum bit
    for bit: random doubles over the whole exponent range, signed zeros,
    subnormals, exact sums, equal and opposite operands and near-cancelling
    ones. A planted mistake (the ordering reversed) must be caught."""
    import numpy as np
    rng = np.random.default_rng(111)
    n = 400_000
    def draw(k):
        kind = rng.integers(0, 6, k)
        v = rng.standard_normal(k) * 10.0 ** rng.uniform(-300, 300, k)
        v = np.where(kind == 0, 0.0, v)
        v = np.where(kind == 1, -0.0, v)
        v = np.where(kind == 2, rng.choice([5e-324, -5e-324, 2.2e-308, -1e-310], k), v)
        v = np.where(kind == 3, np.round(rng.standard_normal(k) * 8) / 8, v)
        return v
    a, b = draw(n), draw(n)
    q = n // 10
    b[:q] = -a[:q] * (1 + rng.standard_normal(q) * 1e-15)
    b[q:2 * q] = a[q:2 * q]
    b[2 * q:3 * q] = -a[2 * q:3 * q]
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    with np.errstate(all="ignore"):
        x = a + b
        bv = x - a
        av = x - bv
        e_ref = (a - av) + (b - bv)
        # the ordering reversed (smaller operand first) must differ somewhere
        small_first = np.abs(a) < np.abs(b)
        xs, ys = np.where(small_first, a, b), np.where(small_first, b, a)
        wrong = ys - ((xs + ys) - xs)
    s, e = np.empty(n), np.empty(n)
    pair_lib.h_two_sum(a.ctypes.data, b.ctypes.data, n, s.ctypes.data, e.ctypes.data)
    assert np.array_equal(s.view(np.uint64), x.view(np.uint64))
    assert np.array_equal(e.view(np.uint64), e_ref.view(np.uint64))
    assert not np.array_equal(wrong.view(np.uint64), e_ref.view(np.uint64))


def test_latitude_searches_on_the_host(pair_lib):
    """The order-preserving integer image of the doubles gives the same search
    results as comparing the values (numpy.searchsorted), on latitude grids,
    random sorted arrays with repeats, and keys on, between and outside the
    values; -0.0 sorts just below +0.0."""
    import numpy as np
    from paper_2510_09892_gb300 import workloads as W
    rng = np.random.default_rng(107)
    arrays = [W.latlon_latitudes(721), W.latlon_latitudes(180),
              np.sort(rng.uniform(-1, 1, 257)),
              np.sort(np.round(rng.uniform(-1, 1, 300), 2)),  # repeats
              np.array([0.5]), np.array([], dtype=np.float64)]
    for a in arrays:
        a = np.ascontiguousarray(a[a != 0.0] if len(a) else a, dtype=np.float64)
        keys = np.concatenate([a, rng.uniform(-1.2, 1.2, 500), np.nextafter(a, 2),
                               np.nextafter(a, -2), [-1.0, 1.0, 0.0, -0.0, np.inf, -np.inf]])
        m = len(keys)
        lower, upper, gallop = (np.empty(m, dtype=np.int64) for _ in range(3))
        pair_lib.h_searches(a.ctypes.data, len(a), keys.ctypes.data, m, lower.ctypes.data,
                            upper.ctypes.data, gallop.ctypes.data)
        assert np.array_equal(lower, np.searchsorted(a, keys, side="left"))
        assert np.array_equal(upper, np.searchsorted(a, keys, side="right"))
        assert np.array_equal(gallop, upper)
    # signed zeros: -0.0 < +0.0 in the image
    a = np.array([-0.5, -0.0, 0.0, 0.5])
    keys = np.array([0.0, -0.0])
    lower, upper, gallop = (np.empty(2, dtype=np.int64) for _ in range(3))
    pair_lib.h_searches(a.ctypes.data, 4, keys.ctypes.data, 2, lower.ctypes.data,
                        upper.ctypes.data, gallop.ctypes.data)
    assert lower.tolist() == [2, 1] and upper.tolist() == [3, 2]


def test_zonal_fixed_point_on_the_host(pair_lib):
    import numpy as np
    from fractions import Fraction as Fr
    rng = np.random.default_rng(108)
    x = np.concatenate([
        rng.standard_normal(2000) * 10.0 ** rng.uniform(-30, 13, 2000),
        [0.0, -0.0, 5e-324, -5e-324, 2.0 ** -81, 3 * 2.0 ** -82, -3 * 2.0 ** -82, 2.0 ** -80,
         2.0 ** 45, -(2.0 ** 46) * 0.999, 2.0 ** 46, np.inf, np.nan]])
    n = len(x)
    lo, hi = np.empty(n, dtype=np.uint64), np.empty(n, dtype=np.uint64)
    ok = np.empty(n, dtype=np.int32)
    pair_lib.h_to_fixed(x.ctypes.data, n, lo.ctypes.data, hi.ctypes.data, ok.ctypes.data)
    values = []
    for i in range(n):
        if not np.isfinite(x[i]) or abs(x[i]) >= 2.0 ** 46:
            assert ok[i] == 0
            continue
        assert ok[i] == 1
        exact = Fr(float(x[i])) * (1 << 80)
        q, r = divmod(abs(exact.numerator), exact.denominator)
        q += 1 if 2 * r >= exact.denominator else 0  # halves away from zero
        want = -q if exact < 0 else q
        got = (int(hi[i]) << 64) | int(lo[i])
        got = got - (1 << 128) if got >> 127 else got
        assert got == want, (x[i], got, want)
        values.append(want)
    # sums of the fixed-point terms (exact integers) back to the nearest double
    sums = [sum(values[:k]) for k in (1, 7, 100, len(values))] + [-(1 << 120) + 12345, (1 << 100) + 1]
    sums += [int(v) for v in rng.integers(-(1 << 62), 1 << 62, 500)]
    m = len(sums)
    lo2 = np.array([s_ & ((1 << 64) - 1) for s_ in sums], dtype=np.uint64)
    hi2 = np.array([(s_ >> 64) & ((1 << 64) - 1) for s_ in sums], dtype=np.uint64)
    out = np.empty(m)
    pair_lib.h_from_fixed(lo2.ctypes.data, hi2.ctypes.data, m, out.ctypes.data)
    for s_, got in zip(sums, out):
        assert got == float(Fr(s_, 1 << 80)), (s_, got)


@pytest.mark.parametrize("axis", [None, 0, 1, 2, "swap"])
def test_accux_intermediates_and_reflections_on_the_host(pair_lib, axis):
    """App. A: the kernel's AccuX built for the host carries exactly the step
    reference's intermediate pairs; and (Sec. 3) reflected or swapped inputs
    give the reflected outputs bit for bit, the slots exchanged where the
    s-term of Eq. 2.2 changes sign."""
    import numpy as np
    from oracle import steps
    from paper_2510_09892_gb300 import workloads as W
    from tests import parity as P
    from tests.test_oracle_steps import _reflect, equal_as_mapped, expected_after
    A, B, z = W.uniform_arcs(3000, seed=109)
    A, B, z = (np.ascontiguousarray(v, dtype=np.float64) for v in (A, B, z))
    n = len(z)

    def run(A_, B_, z_):
        A_, B_, z_ = (np.ascontiguousarray(v, dtype=np.float64) for v in (A_, B_, z_))
        pts = np.empty((n, 2, 3))
        cnt = np.empty(n, dtype=np.int32)
        pair_lib.h_pair_accux(A_.ctypes.data, B_.ctypes.data, z_.ctypes.data, n,
                              pts.ctypes.data, cnt.ctypes.data)
        return cnt, pts

    if axis is None:
        mid = np.empty((n, 16))
        pair_lib.h_accux_mid(A.ctypes.data, B.ctypes.data, z.ctypes.data, n, mid.ctypes.data)
        r = steps.accux_intermediates(A, B, z, variant=2)["raw"]
        ok = r[:, 10] >= 0
        assert P.same_bits(mid[ok, :15], r[ok, :15])
        return
    c0, p0 = run(A, B, z)
    c1, p1 = run(B, A, z) if axis == "swap" else run(*_reflect(A, B, z, axis))
    assert np.array_equal(c0, c1)
    assert equal_as_mapped(c0, p1, expected_after(p0, axis))
