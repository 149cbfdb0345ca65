"""ctypes front end of accux_ref.c (step-by-step FP64 AccuX and direct Eq. 2.2).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
legs may use this module. The shared object is built from accux_ref.c with
plain gcc and -ffp-contract=off (the paper builds its CPU code the same way,
Sec. 7.2), in-tree next to this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "accux_ref.c")
_LIB = os.path.join(_HERE, "liboracle_accux.so")

LITERAL_DOP = 1  # variant bit: AccuDOP with the printed '+' (a planted mistake)

_lib = None


def build(force: bool = False) -> str:
    """Compile accux_ref.c into liboracle_accux.so (idempotent)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        i64 = ctypes.c_int64
        L.oracle_accux.argtypes = [dp, dp, dp, i64, ctypes.c_int, dp, ip]
        L.oracle_direct.argtypes = [dp, dp, dp, i64, dp, ip]
        L.oracle_accux_intermediates.argtypes = [dp, dp, dp, i64, ctypes.c_int, dp]
        L.oracle_two_prod.argtypes = [dp, dp, i64, dp, dp]
        L.oracle_two_sum.argtypes = [dp, dp, i64, dp, dp]
        L.oracle_accu_dop.argtypes = [dp, i64, ctypes.c_int, dp, dp]
        L.oracle_comp_dot_c.argtypes = [dp, dp, i64, ctypes.c_int, dp, dp]
        L.oracle_sum_non_neg.argtypes = [dp, i64, dp, dp]
        L.oracle_sum_of_squares_c.argtypes = [dp, dp, i64, ctypes.c_int, dp, dp]
        L.oracle_acc_sqrt.argtypes = [dp, dp, i64, dp, dp]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _arcs(A, B, z0):
    A, pa = _d(np.asarray(A, dtype=np.float64).reshape(-1, 3))
    B, pb = _d(np.asarray(B, dtype=np.float64).reshape(-1, 3))
    z, pz = _d(np.asarray(z0, dtype=np.float64).reshape(-1))
    if not (A.shape[0] == B.shape[0] == z.shape[0]):
        raise ValueError("A, B, z0 length mismatch")
    return (A, B, z), (pa, pb, pz), z.shape[0]


def accux(A, B, z0, variant: int = 0):
    """Algorithm 8 for both roots: (count int32[n], pts float64[n,2,3])."""
    keep, (pa, pb, pz), n = _arcs(A, B, z0)
    pts = np.empty((n, 2, 3))
    cnt = np.empty(n, dtype=np.int32)
    lib().oracle_accux(pa, pb, pz, n, variant, _d(pts)[1],
                       cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return cnt, pts


def direct(A, B, z0):
    """Direct FP64 Eq. 2.2 for both roots: (count int32[n], pts float64[n,2,3])."""
    keep, (pa, pb, pz), n = _arcs(A, B, z0)
    pts = np.empty((n, 2, 3))
    cnt = np.empty(n, dtype=np.int32)
    lib().oracle_direct(pa, pb, pz, n, _d(pts)[1],
                        cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return cnt, pts


def accux_intermediates(A, B, z0, variant: int = 0):
    """Per-arc intermediates of Algorithm 8 as a dict of arrays (App. A)."""
    keep, (pa, pb, pz), n = _arcs(A, B, z0)
    mid = np.empty((n, 16))
    lib().oracle_accux_intermediates(pa, pb, pz, n, variant, _d(mid)[1])
    return {"n": mid[:, 0:3], "en": mid[:, 3:6], "S2": mid[:, 6], "s2": mid[:, 7],
            "S3": mid[:, 8], "s3": mid[:, 9], "ss2": mid[:, 10], "ess2": mid[:, 11],
            "sb": mid[:, 12], "es": mid[:, 13], "X": mid[:, 14], "raw": mid}


def _pair_out(n):
    p = np.empty(n)
    e = np.empty(n)
    return p, e, _d(p)[1], _d(e)[1]


def two_prod(a, b):
    a, pa = _d(np.asarray(a, dtype=np.float64).reshape(-1))
    b, pb = _d(np.asarray(b, dtype=np.float64).reshape(-1))
    p, e, pp, pe = _pair_out(a.size)
    lib().oracle_two_prod(pa, pb, a.size, pp, pe)
    return p, e


def two_sum(a, b):
    a, pa = _d(np.asarray(a, dtype=np.float64).reshape(-1))
    b, pb = _d(np.asarray(b, dtype=np.float64).reshape(-1))
    p, e, pp, pe = _pair_out(a.size)
    lib().oracle_two_sum(pa, pb, a.size, pp, pe)
    return p, e


def accu_dop(abcd, variant: int = 0):
    """Algorithm 4 on rows (a, b, c, d): pair approximating a*d - b*c."""
    m, pm = _d(np.asarray(abcd, dtype=np.float64).reshape(-1, 4))
    p, e, pp, pe = _pair_out(m.shape[0])
    lib().oracle_accu_dop(pm, m.shape[0], variant, pp, pe)
    return p, e


def comp_dot_c(x, y):
    x, px = _d(np.asarray(x, dtype=np.float64))
    y, py = _d(np.asarray(y, dtype=np.float64))
    n, L = x.shape
    p, e, pp, pe = _pair_out(n)
    lib().oracle_comp_dot_c(px, py, n, L, pp, pe)
    return p, e


def sum_non_neg(AaBb):
    m, pm = _d(np.asarray(AaBb, dtype=np.float64).reshape(-1, 4))
    p, e, pp, pe = _pair_out(m.shape[0])
    lib().oracle_sum_non_neg(pm, m.shape[0], pp, pe)
    return p, e


def sum_of_squares_c(x, e):
    x, px = _d(np.asarray(x, dtype=np.float64))
    e, pe_ = _d(np.asarray(e, dtype=np.float64))
    n, L = x.shape
    S, s, pS, ps = _pair_out(n)
    lib().oracle_sum_of_squares_c(px, pe_, n, L, pS, ps)
    return S, s


def acc_sqrt(S, e):
    S, pS = _d(np.asarray(S, dtype=np.float64).reshape(-1))
    e, pe_ = _d(np.asarray(e, dtype=np.float64).reshape(-1))
    r, er, pr, per = _pair_out(S.size)
    lib().oracle_acc_sqrt(pS, pe_, S.size, pr, per)
    return r, er
