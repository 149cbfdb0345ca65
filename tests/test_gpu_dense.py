"""Parity of the dense CUDA call (sphx_intersect_gca_constlat) with the oracle.

Inputs come from the seeded generators; the expected values come from the
exact-rational oracle (oracle/exact.py) and, for the bit-level checks, from
the step-by-step FP64 reference of the same algorithms (oracle/accux_ref.c),
which performs the same correctly rounded operations in the same order:
  * FP64-EFT (AccuX, Algorithm 8, renormalised AccuDOP) and direct FP64
    (Sec. 4) must equal the step reference bit for bit, counts included;
  * FP64-EFT must match the oracle's hit counts exactly on every arc the oracle
    does not flag as near a boundary, and each point within 4 ulp per
    component (rule in tests/parity.py);
  * float-float must match the counts and stay within its stated bound.
"""
import numpy as np
import pytest
import torch

from oracle import steps
from paper_2510_09892_gb300 import sphx
from paper_2510_09892_gb300 import workloads as W
from tests import parity as P

pytestmark = pytest.mark.gpu



def run(A, B, z, mode):
    dev = torch.device("cuda:0")
    tA = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
    tB = torch.from_numpy(np.ascontiguousarray(B)).to(dev)
    tz = torch.from_numpy(np.ascontiguousarray(z)).to(dev)
    pts = torch.full((len(z), 2, 3), 7.0, dtype=torch.float64, device=dev)  # poison
    cnt = torch.full((len(z),), -99, dtype=torch.int32, device=dev)
    sphx.sphx_intersect_gca_constlat(tA, tB, tz, pts, cnt, mode)
    torch.cuda.synchronize()
    return cnt.cpu().numpy(), pts.cpu().numpy()


def check_against_exact(cnt, pts, A, B, z, ulp_gate=4.0):
    ce, pe, fe = P.run_exact(A, B, z)
    P.assert_unflagged(fe)
    ok = fe == 0
    assert np.array_equal(cnt[ok], ce[ok]), np.flatnonzero((cnt != ce) & ok)[:10]
    hit = np.isfinite(pe[..., 0]) & ok[:, None]
    assert np.array_equal(np.isfinite(pts[..., 0]) & ok[:, None], hit)
    _, _, gate = P.component_errors(pts, pe, z)
    worst = np.nanmax(np.where(hit[..., None], gate, 0.0))
    assert worst <= ulp_gate, worst
    return ce, pe, fe


@pytest.mark.parametrize("n", [1, 5, 127, 128, 129, 1000, 10_000])
def test_eft_uniform_bit_exact_and_within_4ulp(n):
    A, B, z = W.uniform_arcs(n, seed=100 + n)
    cnt, pts = run(A, B, z, "eft")
    cr, pr = steps.accux(A, B, z, variant=2)
    assert np.array_equal(cnt, cr)
    assert P.same_bits(pts, pr)
    check_against_exact(cnt, pts, A, B, z)


def test_direct_uniform_bit_exact_with_step_reference():
    A, B, z = W.uniform_arcs(10_000)
    cnt, pts = run(A, B, z, "direct")
    cr, pr = steps.direct(A, B, z)
    assert np.array_equal(cnt, cr)
    assert P.same_bits(pts, pr)


def test_printed_variant_bit_exact_with_step_reference():
    A, B, z = W.stress_arcs(5000, seed=7)
    cnt, pts = run(A, B, z, "eft_printed")
    cr, pr = steps.accux(A, B, z, variant=0)
    assert np.array_equal(cnt, cr)
    assert P.same_bits(pts, pr)


def test_eft_stress_mix_within_4ulp_and_direct_worse():
    A, B, z, k = W.stress_arcs(20_000, seed=11, return_class=True)
    cnt, pts = run(A, B, z, "eft")
    cr, pr = steps.accux(A, B, z, variant=2)
    assert np.array_equal(cnt, cr) and P.same_bits(pts, pr)
    ce, pe, fe = check_against_exact(cnt, pts, A, B, z)
    # the paper's norm metric stays within its bound 3 sqrt(1 - z0^2) u (Sec. 6.2)
    ok = (fe == 0)[:, None] & np.isfinite(pe[..., 0])
    assert np.nanmax(np.where(ok, P.norm_error(pts, pe, z), 0)) <= 3.0
    # direct FP64 loses about half the digits on this mix (Sec. 4)
    cd, pd = run(A, B, z, "direct")
    both = ok & np.isfinite(pd[..., 0])
    assert np.nanmax(np.where(both, P.norm_error(pd, pe, z), 0)) > 1e3


def gen_arcs(gen):
    """Well-conditioned, ill-conditioned, mixed and non-unit seeded inputs."""
    if gen == "uniform":
        return W.uniform_arcs(10_000, seed=41)
    if gen == "stress":
        return W.stress_arcs(40_000, seed=42)
    if gen == "mixed":
        return W.mixed_chunk(7, size=20_000)
    # endpoints scaled by 10^+-30: the formula only uses directions
    A, B, z = W.stress_arcs(20_000, seed=43)
    rng = np.random.default_rng(44)
    A = A * (10.0 ** rng.uniform(-30, 30, len(z)))[:, None]
    B = B * (10.0 ** rng.uniform(-30, 30, len(z)))[:, None]
    return A, B, z


@pytest.mark.parametrize("gen", ["uniform", "stress", "mixed", "scaled"])
def test_wide_int_matches_exact_oracle(gen):
    """The integer-limb evaluation: exact hit counts on unflagged arcs and
    every coordinate within 1 ulp of the correctly rounded exact value (the
    4-ulp bound with room to spare: 96-bit mantissas leave the rounding to
    decide), on well-conditioned, ill-conditioned, mixed and non-unit inputs."""
    A, B, z = gen_arcs(gen)
    cnt, pts = run(A, B, z, "wide")
    ce, pe, fe = check_against_exact(cnt, pts, A, B, z, ulp_gate=1.0)
    ok = (fe == 0)[:, None] & np.isfinite(pe[..., 0])
    assert np.nanmax(np.where(ok, P.norm_error(pts, pe, z), 0)) <= 1.0


def test_wide_int_full_size_stress_sampled():
    """The 10^6-arc stress workload in the benchmark's launch shape, a seeded
    sample of 20 000 arcs against the exact oracle; on all arcs the wide
    evaluation and FP64-EFT agree on the hit counts wherever neither is near
    a boundary, and their points within the sum of their bounds."""
    A, B, z = W.stress_arcs(1_000_000)
    cnt, pts = run(A, B, z, "wide")
    idx = np.sort(np.random.default_rng(3).choice(len(z), 20_000, replace=False))
    check_against_exact(cnt[idx], pts[idx], A[idx], B[idx], z[idx], ulp_gate=1.0)
    ce, pe = run(A, B, z, "eft")
    same = cnt == ce
    assert same.mean() > 0.999
    both = np.isfinite(pts[..., 0]) & np.isfinite(pe[..., 0]) & same[:, None]
    _, _, gate = P.component_errors(pe, pts, z)
    assert np.nanmax(np.where(both[..., None], gate, 0)) <= 5.0


def run_adaptive(A, B, z, fallback=None, gate=4.0):
    dev = torch.device("cuda:0")
    tA, tB, tz = (torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (A, B, z))
    pts = torch.full((len(z), 2, 3), 7.0, dtype=torch.float64, device=dev)  # poison
    cnt = torch.full((len(z),), -99, dtype=torch.int32, device=dev)
    fb = torch.zeros(1, dtype=torch.int64, device=dev) if fallback is None else fallback
    sphx.sphx_intersect_gca_constlat_adaptive(tA, tB, tz, pts, cnt, gate, fb)
    torch.cuda.synchronize()
    return cnt.cpu().numpy(), pts.cpu().numpy(), int(fb.item())


def check_adaptive(gen, gate):
    """Every arc within the gate and with the exact hit count on unflagged
    arcs. Arcs the filter hands on are evaluated by the integer-limb form, so
    an arc whose result differs from that form in any bit was kept by the
    filter: those must have the exact hit count even where the oracle flags a
    near-boundary case, and their number cannot exceed the arcs the filter
    kept. Returns the share of arcs the filter kept."""
    A, B, z = gen_arcs(gen)
    cnt, pts, fb = run_adaptive(A, B, z, gate=gate)
    cw, pw = run(A, B, z, "wide")
    ce, pe, fe = check_against_exact(cnt, pts, A, B, z, ulp_gate=gate)
    bits = lambda p: np.where(np.isnan(p), 0.0, p).view(np.int64)
    kept = (cnt != cw) | (bits(pts) != bits(pw)).any(axis=(1, 2))
    assert 0 <= fb <= len(z) and kept.sum() <= len(z) - fb
    assert np.array_equal(cnt[kept], ce[kept])
    hit = np.isfinite(pe[kept][..., 0])
    _, _, g = P.component_errors(pts[kept], pe[kept], z[kept])
    assert np.nanmax(np.where(hit[..., None], g, 0.0), initial=0.0) <= gate
    share = 1 - fb / len(z)
    print(f"{gen}, gate {gate:g} ulp: filter kept {share:.3f} of {len(z)} arcs, "
          f"{kept.mean():.3f} differ from the integer-limb result")
    return share


@pytest.mark.parametrize("gen", ["uniform", "stress", "mixed", "scaled"])
def test_adaptive_filter_within_4ulp(gen):
    """The adaptive mode at its own gate (4 ulp per component)."""
    check_adaptive(gen, 4.0)


@pytest.mark.parametrize("gen,gate,min_kept", [("uniform", 64.0, 0.3), ("mixed", 64.0, 0.2),
                                               ("stress", 2.0 ** 20, 0.08)])
def test_adaptive_filter_relaxed_gates(gen, gate, min_kept):
    """Looser gates let the filter keep many arcs, which tests its bound: the
    kept arcs of well-conditioned and of ill-conditioned inputs must keep
    exact hit counts and stay within the gate against the exact oracle."""
    assert check_adaptive(gen, gate) >= min_kept


def test_adaptive_fallback_counter_accumulates():
    A, B, z = W.stress_arcs(3000, seed=17)
    fb = torch.zeros(1, dtype=torch.int64, device=torch.device("cuda:0"))
    c1, p1, f1 = run_adaptive(A, B, z, fb)
    c2, p2, f2 = run_adaptive(A, B, z, fb)
    assert 0 < f1 <= len(z) and f2 == 2 * f1
    assert np.array_equal(c1, c2) and P.same_bits(p1, p2)
    # the plain dense call in the adaptive mode gives the same results
    c3, p3 = run(A, B, z, "adaptive")
    assert np.array_equal(c1, c3) and P.same_bits(p1, p3)


@pytest.mark.parametrize("gen", ["uniform", "stress", "mixed", "scaled"])
def test_ff32_within_stated_bound(gen):
    """Float-float: |dP| <= 2^-44 sqrt(1 - z0^2) on every unflagged hit, near
    tangency and the poles included (its cancelling steps are exact or
    128-bit), and the exact oracle's hit counts on every unflagged arc."""
    A, B, z = gen_arcs(gen)
    cnt, pts = run(A, B, z, "ff32")
    ce, pe, fe = P.run_exact(A, B, z)
    P.assert_unflagged(fe)
    ok = fe == 0
    assert np.array_equal(cnt[ok], ce[ok]), np.flatnonzero((cnt != ce) & ok)[:10]
    hit = np.isfinite(pe[..., 0]) & ok[:, None]
    assert np.array_equal(np.isfinite(pts[..., 0]) & ok[:, None], hit)
    err = P.norm_error(pts, pe, z)
    worst = np.nanmax(np.where(hit, err, 0))
    print(f"\nff32 {gen}: worst |dP| = {worst / P.FF_BOUND:.3f} of the stated bound")
    assert worst <= P.FF_BOUND


def test_edge_cases():
    nan, inf = float("nan"), float("inf")
    e = np.array([1.0, 0.0, 0.0])
    rows = [
        # (x1, x2, z0, expected count)
        (e, e, 0.3, -1),                                  # x1 == x2: n = 0
        (e, -e, 0.0, -1),                                 # antipodal: n = 0
        (e, [0.0, 1.0, 0.0], 0.0, -1),                    # on the equator, z0 = 0
        (e, [0.0, 1.0, 0.0], 0.5, 0),                     # on the equator, z0 != 0
        ([nan, 0, 1], e, 0.1, 0),                         # NaN input
        (e, [0.0, 0.0, 1.0], inf, 0),                     # infinite z0
        ([0.6, 0.0, 0.8], [0.0, 0.6, 0.8], 0.8, 2),       # both endpoints on the latitude
        ([0.6, 0.0, 0.8], [0.0, 0.6, 0.8], 0.9, 0),       # above the great circle's top
        ([1.0, 0.0, 0.0], [0.0, 0.0, 1.0], 1.0, 1),       # meridian arc to the pole: tangent at the pole
        ([1.0, 0.0, 0.0], [0.0, 0.0, 1.0], 0.0, 1),       # meridian arc through the equator endpoint
        ([2.0, 0.0, 0.0], [0.0, 0.0, 3.0], 0.5, 1),       # non-unit endpoints
    ]
    A = np.array([r[0] for r in rows], dtype=np.float64)
    B = np.array([r[1] for r in rows], dtype=np.float64)
    z = np.array([r[2] for r in rows], dtype=np.float64)
    from oracle import exact
    want = np.array([exact.intersect(A[i], B[i], z[i]).count for i in range(len(z))])
    for mode in ("eft", "direct", "ff32", "wide", "adaptive"):
        cnt, pts = run(A, B, z, mode)
        # degenerate, non-finite and equator cases are exact decisions in every mode
        assert np.array_equal(cnt[:6], want[:6]), (mode, cnt, want)
        assert np.isnan(pts[:6]).all()
        # exactly max(count, 0) slots hold a point, the others are NaN
        filled = np.isfinite(pts).all(axis=2).sum(axis=1)
        assert np.array_equal(filled, np.maximum(cnt, 0))
        assert (np.isfinite(pts).all(axis=2) | np.isnan(pts).all(axis=2)).all()
    for mode in ("eft", "wide", "adaptive"):
        cnt, pts = run(A, B, z, mode)
        assert np.array_equal(cnt, want), mode


def test_n_zero_and_bad_arguments():
    dev = torch.device("cuda:0")
    z = torch.zeros(0, dtype=torch.float64, device=dev)
    A = torch.zeros((0, 3), dtype=torch.float64, device=dev)
    pts = torch.zeros((0, 2, 3), dtype=torch.float64, device=dev)
    cnt = torch.zeros(0, dtype=torch.int32, device=dev)
    sphx.sphx_intersect_gca_constlat(A, A, z, pts, cnt, "eft")  # no-op
    L = sphx.lib()
    A = torch.zeros((64, 3), dtype=torch.float64, device=dev)
    z = torch.zeros(64, dtype=torch.float64, device=dev)
    pts = torch.zeros((64, 2, 3), dtype=torch.float64, device=dev)
    cnt = torch.zeros(64, dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream().cuda_stream
    p = A.data_ptr()
    assert L.sphx_intersect_gca_constlat(p, p, z.data_ptr(), 64, pts.data_ptr(), cnt.data_ptr(),
                                         9, s) == sphx.ERR_INVALID_ARG
    assert L.sphx_intersect_gca_constlat(p + 8, p, z.data_ptr(), 63, pts.data_ptr(),
                                         cnt.data_ptr(), 1, s) == sphx.ERR_INVALID_ARG
    assert L.sphx_intersect_gca_constlat(p, p, z.data_ptr(), -1, pts.data_ptr(), cnt.data_ptr(),
                                         1, s) == sphx.ERR_INVALID_ARG
    torch.cuda.synchronize()


def test_graph_capture_replays_dense_call():
    A, B, z = W.uniform_arcs(4096, seed=5)
    dev = torch.device("cuda:0")
    tA, tB, tz = (torch.from_numpy(v).to(dev) for v in (A, B, z))
    pts = torch.empty((4096, 2, 3), dtype=torch.float64, device=dev)
    cnt = torch.empty(4096, dtype=torch.int32, device=dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        sphx.sphx_intersect_gca_constlat(tA, tB, tz, pts, cnt, "eft", s)  # warm-up
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sphx.sphx_intersect_gca_constlat(tA, tB, tz, pts, cnt, "eft", s)
    pts.fill_(0)
    g.replay()
    torch.cuda.synchronize()
    cr, pr = steps.accux(A, B, z, variant=2)
    assert np.array_equal(cnt.cpu().numpy(), cr)
    assert P.same_bits(pts.cpu().numpy(), pr)


def test_full_size_stress_workload_sampled():
    """The 10^6-arc ill-conditioned workload in the benchmark's launch shape:
    every arc bit-exact with the step reference, a seeded sample of 20 000
    arcs against the exact oracle."""
    A, B, z = W.stress_arcs(1_000_000)
    cnt, pts = run(A, B, z, "eft")
    cr, pr = steps.accux(A, B, z, variant=2)
    assert np.array_equal(cnt, cr)
    assert P.same_bits(pts, pr)
    idx = np.sort(np.random.default_rng(0).choice(len(z), 20_000, replace=False))
    check_against_exact(cnt[idx], pts[idx], A[idx], B[idx], z[idx])
    cd, pd = run(A, B, z, "direct")
    cr, pr = steps.direct(A, B, z)
    assert np.array_equal(cd, cr) and P.same_bits(pd, pr)


@pytest.mark.parametrize("n", [1, 1_000, 393_217, 1_572_865, 8_519_681])
@pytest.mark.parametrize("pinned", ["all", "none", "inputs"])
def test_host_buffer_call_equals_device_call(n, pinned):
    """sphx_intersect_gca_constlat_host: with every buffer page-locked the
    kernel works on host memory in place; otherwise (pageable, or only the
    inputs page-locked) four chunks (more past 4 x 2^21 arcs: 8 519 681 takes
    five, the last one short) go through the context's staging. Identical
    results to the device-buffer call either way, uneven chunks included."""
    A, B, z = W.stress_arcs(n, seed=50 + n % 7)
    cnt_d, pts_d = run(A, B, z, "wide")
    hA, hB, hz = (torch.from_numpy(np.ascontiguousarray(v)) for v in (A, B, z))
    hP = torch.full((n, 2, 3), 5.0, dtype=torch.float64)
    hC = torch.full((n,), -9, dtype=torch.int32)
    if pinned == "all":
        hA, hB, hz, hP, hC = (t.pin_memory() for t in (hA, hB, hz, hP, hC))
    elif pinned == "inputs":
        hA, hB, hz = (t.pin_memory() for t in (hA, hB, hz))
    with sphx.Context(0) as ctx:
        for _ in range(2):  # the second call reuses the staging
            sphx.sphx_intersect_gca_constlat_host(ctx, hA, hB, hz, hP, hC, "wide")
            sphx.sphx_host_join(ctx)
            torch.cuda.synchronize()
            assert np.array_equal(hC.numpy(), cnt_d)
            assert P.same_bits(hP.numpy(), pts_d)
            hP.fill_(5.0)
            hC.fill_(-9)


@pytest.mark.parametrize("pinned", ["all", "none"])
def test_host_buffer_call_adaptive_mode(pinned):
    """The adaptive mode through the host-buffer call (in place, and through the
    staged copies) equals the device call bit for bit."""
    A, B, z = W.mixed_chunk(3, size=50_001)
    cnt_d, pts_d = run(A, B, z, "adaptive")
    hA, hB, hz = (torch.from_numpy(np.ascontiguousarray(v)) for v in (A, B, z))
    hP = torch.full((len(z), 2, 3), 5.0, dtype=torch.float64)
    hC = torch.full((len(z),), -9, dtype=torch.int32)
    if pinned == "all":
        hA, hB, hz, hP, hC = (t.pin_memory() for t in (hA, hB, hz, hP, hC))
    with sphx.Context(0) as ctx:
        sphx.sphx_intersect_gca_constlat_host(ctx, hA, hB, hz, hP, hC, "adaptive")
        sphx.sphx_host_join(ctx)
        torch.cuda.synchronize()
    assert np.array_equal(hC.numpy(), cnt_d)
    assert P.same_bits(hP.numpy(), pts_d)


def test_host_buffer_calls_overlap_and_join():
    """Successive host-buffer calls on one context, different batches, one
    join at the end: every call's outputs are complete and correct."""
    batches = [W.uniform_arcs(200_003, seed=60 + k) for k in range(3)]
    want = [run(A, B, z, "wide") for A, B, z in batches]
    outs = []
    with sphx.Context(0) as ctx:
        for A, B, z in batches:
            hA, hB, hz = (torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for v in (A, B, z))
            hP = torch.empty((len(z), 2, 3), dtype=torch.float64).pin_memory()
            hC = torch.empty(len(z), dtype=torch.int32).pin_memory()
            sphx.sphx_intersect_gca_constlat_host(ctx, hA, hB, hz, hP, hC, "wide")
            outs.append((hA, hB, hz, hP, hC))
        sphx.sphx_host_join(ctx)
        torch.cuda.synchronize()
    for (cnt, pts), (_, _, _, hP, hC) in zip(want, outs):
        assert np.array_equal(hC.numpy(), cnt)
        assert P.same_bits(hP.numpy(), pts)


def test_accux_intermediates_equal_step_reference():
    """sphx_accux_intermediates (App. A) dumps exactly the pairs the step
    reference carries, for every arc with a candidate."""
    A, B, z = W.uniform_arcs(20_000, seed=71)
    dev = torch.device("cuda:0")
    tA, tB, tz = (torch.from_numpy(v).to(dev) for v in (A, B, z))
    mid = torch.empty((len(z), 16), dtype=torch.float64, device=dev)
    sphx.sphx_accux_intermediates(tA, tB, tz, mid)
    torch.cuda.synchronize()
    g = mid.cpu().numpy()
    r = steps.accux_intermediates(A, B, z, variant=2)["raw"]
    ok = r[:, 10] >= 0  # arcs with candidates (s^2 >= 0): the whole chain ran
    assert P.same_bits(g[ok, :15], r[ok, :15])


@pytest.mark.parametrize("mode", ["wide", "eft", "direct", "ff32"])
@pytest.mark.parametrize("axis", [0, 1, 2, "swap"])
def test_reflection_equivariance_on_gpu(mode, axis):
    """Reflected inputs give the reflected outputs bit for bit (slots exchanged
    where the s-term of Eq. 2.2 changes sign): the reduction of Sec. 3 holds
    exactly for every mode."""
    from tests.test_oracle_steps import _reflect, equal_as_mapped, expected_after
    A, B, z = W.stress_arcs(20_000, seed=72)
    c0, p0 = run(A, B, z, mode)
    if axis == "swap":
        c1, p1 = run(B, A, z, mode)
    else:
        c1, p1 = run(*_reflect(A, B, z, axis), mode)
    assert np.array_equal(c0, c1)
    assert equal_as_mapped(c0, p1, expected_after(p0, axis))


def test_error_distribution_report():
    """Error distributions against the exact oracle, per mode and workload
    (printed; run with -s to see them): the fraction of coordinates that are
    correctly rounded, and the median / p95 / p99 / max of the component
    error in the gate's units (ulp for large components, u sqrt(1 - z0^2) for
    small ones), over unflagged arcs. Bounds: integer limbs <= 1, FP64-EFT
    <= 4; direct FP64 loses many digits on the stress mix (Sec. 4)."""
    rows = []
    for name, (A, B, z) in (("uniform", W.uniform_arcs(20_000, seed=14)),
                            ("stress", W.stress_arcs(20_000, seed=13))):
        ce, pe, fe = P.run_exact(A, B, z)
        P.assert_unflagged(fe)
        ok = fe == 0
        for mode in ("wide", "eft", "direct", "ff32"):
            cnt, pts = run(A, B, z, mode)
            both = ok[:, None] & np.isfinite(pe[..., 0]) & np.isfinite(pts[..., 0])
            ulp, _, gate = P.component_errors(pts, pe, z)
            g = gate[both]
            exact_frac = float(np.mean(ulp[both] == 0.0))
            q = np.percentile(g, [50, 95, 99])
            counts_equal = float(np.mean(cnt[ok] == ce[ok]))
            rows.append((name, mode, exact_frac, q[0], q[1], q[2], float(g.max()), counts_equal))
            if mode == "wide":
                assert g.max() <= 1.0 and exact_frac > 0.999
            if mode == "eft":
                assert g.max() <= 4.0
            if mode == "direct" and name == "stress":
                assert g.max() > 100.0
            if mode in ("wide", "eft"):
                assert counts_equal == 1.0
    print("\nworkload  mode    correctly-rounded  p50     p95     p99     max        counts")
    for r in rows:
        print(f"{r[0]:9s} {r[1]:7s} {r[2]:17.6f}  {r[3]:.3g}  {r[4]:.3g}  {r[5]:.3g}  {r[6]:.4g}  {r[7]:.6f}")
