"""Error metrics and oracle runners shared by the parity tests (no method arithmetic).

Error rule for "<= 4 ulp per component" (the paper bounds only |dP|, Sec. 1.2,
and notes that a coordinate's relative error is undefined where it vanishes):
  * a component c with |P_c| >= 2^-20 sqrt(1 - z0^2) is gated on
    |P~_c - P_c| / ulp(P_c) <= 4, ulp taken of the correctly rounded exact value;
  * a smaller component is gated on the absolute error |P~_c - P_c| <= 4 u sqrt(1 - z0^2),
    u = 2^-53 (it comes out of a cancelling compensated dot product).
The norm metric of Sec. 1.2, |P~ - P| / (u sqrt(1 - z0^2)), is reported beside it.
"""
from __future__ import annotations

import os

import numpy as np

U = 2.0 ** -53
SMALL_COMPONENT = 2.0 ** -20


def ulp_of(x):
    """ulp of each finite double: 2^(exponent - 52), with the subnormal floor."""
    x = np.abs(np.asarray(x, dtype=np.float64))
    m, e = np.frexp(x)  # x = m 2^e, m in [0.5, 1)
    return np.ldexp(np.ones_like(x), np.maximum(e - 53, -1074))


def component_errors(pts, ref, z0):
    """Per-component error in units of the gate: (ulp_err, abs_err_units, gated_value).

    pts, ref: (n, 2, 3). Returns arrays (n, 2, 2) for the x and y components:
    the gate value is ulp error for large components and absolute error in units
    of u sqrt(1 - z0^2) for small ones; both must be <= 4.
    """
    rho = np.sqrt(np.maximum(0.0, (1.0 - z0) * (1.0 + z0)))[:, None, None]
    p = pts[..., :2]
    r = ref[..., :2]
    d = np.abs(p - r)
    with np.errstate(invalid="ignore", divide="ignore"):
        ulp_err = d / ulp_of(r)
        abs_err = d / (U * rho)
    large = np.abs(r) >= SMALL_COMPONENT * rho
    gate = np.where(large, ulp_err, abs_err)
    return ulp_err, abs_err, gate


def norm_error(pts, ref, z0):
    """|P~ - P| / (u sqrt(1 - z0^2)) per slot (Sec. 1.2 metric)."""
    rho = np.sqrt(np.maximum(0.0, (1.0 - z0) * (1.0 + z0)))[:, None]
    d = pts - ref
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.sqrt(d[..., 0] ** 2 + d[..., 1] ** 2) / (U * rho)


# float-float's stated bound: the cancelling steps (n, |n_xy|^2, s^2) are
# exact or 128-bit on integer limbs, the rest runs on FP32 pairs (2^-48), and
# |P~ - P| <= 2^-44 sqrt(1 - z0^2) on every arc; in the norm_error unit
# (u sqrt(1 - z0^2)) that is 2^-44 / 2^-53 = 512
FF_BOUND = 2.0 ** -44 / U


# Every exact comparison skips the arcs the oracle flags as near a boundary;
# this floor keeps over-flagging from hollowing those comparisons out. The
# seeded uniform, stress and mixed workloads carry at most ~0.06 % flagged
# arcs (near-endpoint short arcs of the stress mix).
MIN_UNFLAGGED = 0.999


def assert_unflagged(flags, min_share=MIN_UNFLAGGED):
    """Assert that at least min_share of the oracle's results carry no flag;
    returns the unflagged share."""
    flags = np.asarray(flags)
    if flags.size == 0:
        return 1.0
    share = float(np.mean(flags == 0))
    assert share >= min_share, f"only {share:.5f} of the cases are unflagged (< {min_share})"
    return share


def hit_mask(count, pts):
    return np.isfinite(pts[..., 0])


def oracle_processes() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def run_exact(A, B, z0):
    """The exact oracle over a batch, in a spawn pool (safe after CUDA started)."""
    from oracle import exact
    return exact.intersect_batch(A, B, z0, processes=oracle_processes())


def same_bits(a, b) -> bool:
    """Bitwise equality of float arrays (NaN payloads compared as NaN)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    both_nan = np.isnan(a) & np.isnan(b)
    return bool(np.all(both_nan | (a.view(np.int64) == b.view(np.int64))))
