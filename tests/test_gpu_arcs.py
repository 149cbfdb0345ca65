"""Parity of the arc x arc CUDA call (sphx_intersect_gca_gca) with the exact
oracle (oracle/exact_arcs.py): hit counts exact on every pair the oracle does
not flag as near a boundary; points within 1 ulp per component for the
integer-limb form and 4 ulp for the FP64-EFT form (the small-component rule of
tests/parity.py, with |p| = 1 as the scale); the direct FP64 form reported."""
import numpy as np
import pytest
import torch

from oracle import exact_arcs as X
from paper_2510_09892_gb300 import sphx
from paper_2510_09892_gb300 import workloads as W
from tests import parity as P

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def run(A1, A2, B1, B2, mode):
    t = [torch.from_numpy(np.ascontiguousarray(v)).to(DEV) for v in (A1, A2, B1, B2)]
    n = t[0].shape[0]
    pts = torch.full((n, 2, 3), 3.0, dtype=torch.float64, device=DEV)  # poisoned
    cnt = torch.full((n,), -77, dtype=torch.int32, device=DEV)
    sphx.sphx_intersect_gca_gca(*t, pts, cnt, mode)
    torch.cuda.synchronize()
    return cnt.cpu().numpy(), pts.cpu().numpy()


def gate(pts, ref):
    """Per-component error: ulps for |p_c| >= 2^-20, absolute in u otherwise."""
    d = np.abs(pts - ref)
    with np.errstate(invalid="ignore", divide="ignore"):
        g = np.where(np.abs(ref) >= 2.0 ** -20, d / P.ulp_of(ref), d / P.U)
    return g


def check(A1, A2, B1, B2, mode, ulps):
    cnt, pts = run(A1, A2, B1, B2, mode)
    ce, pe, fe = X.intersect_arcs_batch(A1, A2, B1, B2, processes=P.oracle_processes())
    # a tenth of the pairs cross within 1e-12..1e-3 of an endpoint on purpose
    P.assert_unflagged(fe, 0.99)
    ok = fe == 0
    assert np.array_equal(cnt[ok], ce[ok]), np.flatnonzero((cnt != ce) & ok)[:10]
    hit = np.isfinite(pe[..., 0]) & ok[:, None]
    assert np.array_equal(np.isfinite(pts[..., 0]) & ok[:, None], hit)
    g = np.where(hit[..., None], gate(pts, pe), 0.0)
    assert np.nanmax(g) <= ulps, np.nanmax(g)
    return cnt, pts, ce, pe, fe


@pytest.mark.parametrize("mode,ulps", [("wide", 1.0), ("eft", 4.0)])
@pytest.mark.parametrize("n", [1, 127, 129, 20_000])
def test_arc_pairs_against_exact(mode, ulps, n):
    A1, A2, B1, B2 = W.arc_pairs(n, seed=200 + n)
    check(A1, A2, B1, B2, mode, ulps)


def test_wide_with_non_unit_endpoints():
    A1, A2, B1, B2 = W.arc_pairs(10_000, seed=211)
    rng = np.random.default_rng(212)
    sc = [(10.0 ** rng.uniform(-30, 30, len(A1)))[:, None] for _ in range(4)]
    check(A1 * sc[0], A2 * sc[1], B1 * sc[2], B2 * sc[3], "wide", 1.0)


def test_direct_counts_on_well_conditioned_pairs():
    A1, A2, B1, B2, k = W.arc_pairs(20_000, seed=213, return_class=True)
    cnt, pts = run(A1, A2, B1, B2, "direct")
    ce, pe, fe = X.intersect_arcs_batch(A1, A2, B1, B2, processes=P.oracle_processes())
    P.assert_unflagged(fe[k == 0])
    uni = (k == 0) & (fe == 0)
    assert (cnt[uni] == ce[uni]).mean() > 0.999
    # direct FP64 loses accuracy on short and nearly parallel arcs
    bad = (k == 1) | (k == 2)
    both = np.isfinite(pe[..., 0]) & np.isfinite(pts[..., 0]) & (fe == 0)[:, None] & bad[:, None]
    assert np.nanmax(np.where(both[..., None], gate(pts, pe), 0)) > 1e3


def test_edge_cases_all_modes():
    e, f, g = (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)
    nan = float("nan")
    rows = [
        (e, e, f, g),                           # arc a degenerate
        (e, f, (0.0, 2.0, 0.0), (3.0, 0.0, 0.0)),  # same great circle
        ((nan, 0.0, 0.0), f, e, g),             # non-finite
        (e, f, (-1.0, -1.0, -1.0), (-1.0, -1.0, 1.0)),  # circles cross, arcs do not
        (e, f, (3.0, 4.0, -5.0), (3.0, 4.0, 5.0)),      # crossing at (0.6, 0.8, 0)
    ]
    A1, A2, B1, B2 = (np.array([r[i] for r in rows]) for i in range(4))
    want = [X.intersect_arcs(*r).count for r in rows]
    assert want == [-1, -1, 0, 0, 1]
    for mode in ("wide", "eft", "direct"):
        cnt, pts = run(A1, A2, B1, B2, mode)
        assert list(cnt) == want, mode
        assert np.isnan(pts[:4]).all()
    cnt, pts = run(A1, A2, B1, B2, "wide")
    assert pts[4, 0].tolist() == [0.6, 0.8, 0.0] and np.isnan(pts[4, 1]).all()


def test_bad_arguments():
    L = sphx.lib()
    t = torch.zeros((64, 3), dtype=torch.float64, device=DEV)
    pts = torch.zeros((64, 2, 3), dtype=torch.float64, device=DEV)
    cnt = torch.zeros(64, dtype=torch.int32, device=DEV)
    p = t.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    assert L.sphx_intersect_gca_gca(p, p, p, p, 64, pts.data_ptr(), cnt.data_ptr(),
                                    sphx.MODE_EFT_FF32, s) == sphx.ERR_UNSUPPORTED
    assert L.sphx_intersect_gca_gca(p + 8, p, p, p, 63, pts.data_ptr(), cnt.data_ptr(),
                                    sphx.MODE_WIDE_INT, s) == sphx.ERR_INVALID_ARG
    assert L.sphx_intersect_gca_gca(p, p, p, p, -1, pts.data_ptr(), cnt.data_ptr(),
                                    sphx.MODE_WIDE_INT, s) == sphx.ERR_INVALID_ARG
    assert L.sphx_intersect_gca_gca(p, p, p, p, 0, pts.data_ptr(), cnt.data_ptr(),
                                    sphx.MODE_WIDE_INT, s) == sphx.OK


def test_full_size_arc_pairs_sampled():
    """The 10^6-pair arc workload in the benchmark's launch shape: a seeded
    sample of 20 000 pairs against the exact oracle; on all pairs, the
    integer-limb and EFT forms agree on the counts and every hit is a unit
    vector lying on its arcs' plane to rounding."""
    A1, A2, B1, B2, k = W.arc_pairs(1_000_000, return_class=True)
    cw, pw = run(A1, A2, B1, B2, "wide")
    idx = np.sort(np.random.default_rng(5).choice(len(A1), 20_000, replace=False))
    ce, pe, fe = X.intersect_arcs_batch(A1[idx], A2[idx], B1[idx], B2[idx],
                                        processes=P.oracle_processes())
    P.assert_unflagged(fe, 0.99)
    P.assert_unflagged(fe[k[idx] != 3])  # all but the near-endpoint class
    ok = fe == 0
    assert np.array_equal(cw[idx][ok], ce[ok])
    hit = np.isfinite(pe[..., 0]) & ok[:, None]
    assert np.nanmax(np.where(hit[..., None], gate(pw[idx], pe), 0)) <= 1.0
    cf, pf = run(A1, A2, B1, B2, "eft")
    assert (cw == cf).mean() > 0.999
    h = np.isfinite(pw[..., 0])
    r2 = (pw ** 2).sum(-1)[h]
    assert np.abs(r2 - 1).max() < 1e-14
    # on arc a's plane, checked where a plain FP64 normal is itself accurate:
    # arcs longer than 0.1 rad (short arcs' plain normals are not)
    na = np.cross(A1, A2)
    long_a = np.linalg.norm(A1 - A2, axis=1) > 0.1
    na /= np.linalg.norm(na, axis=1, keepdims=True)
    dot = np.abs((pw * na[:, None, :]).sum(-1))[h & long_a[:, None]]
    assert dot.max() < 1e-14
