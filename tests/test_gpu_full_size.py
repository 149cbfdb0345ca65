"""Parity at full size: the 2 x 10^8-arc mixed workload (90 % uniform, 10 %
ill-conditioned) in one launch per mode, checked

  * on every arc, on the GPU, by properties that hold at any size: hit counts
    in {0, 1, 2}, every hit on the unit sphere at its latitude, the integer-limb
    and FP64-EFT evaluations agreeing on the hit counts wherever neither is
    near a boundary and on the points within the sum of their bounds;
  * on a seeded sample of 10^5 arcs spread over the whole batch, against
    the exact-rational oracle (exact hit counts on unflagged arcs, <= 1 ulp
    for the integer-limb form, <= 4 ulp for FP64-EFT, the stated bound for
    float-float), with each mode's 95th-percentile and maximum error printed
    beside direct FP64's (run with -s).

The chunks of the mixed workload are seeded independently, so they are
generated in parallel (a 'spawn' pool) and copied to the device one by one.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest
import torch

from paper_2510_09892_gb300 import sphx
from paper_2510_09892_gb300 import workloads as W
from tests import parity as P

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
N_FULL = 200_000_000
N_SAMPLE = 100_000


@pytest.fixture(scope="module")
def full_batch():
    n = N_FULL
    tA = torch.empty((n, 3), dtype=torch.float64, device=DEV)
    tB = torch.empty((n, 3), dtype=torch.float64, device=DEV)
    tz = torch.empty(n, dtype=torch.float64, device=DEV)
    rng = np.random.default_rng(2024)
    sample = np.sort(rng.choice(n, N_SAMPLE, replace=False))
    sA = np.empty((N_SAMPLE, 3))
    sB = np.empty((N_SAMPLE, 3))
    sz = np.empty(N_SAMPLE)
    nchunks = (n + W.CHUNK - 1) // W.CHUNK
    procs = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        for k, (A, B, z) in enumerate(pool.imap(W.mixed_chunk, range(nchunks))):
            lo, hi = k * W.CHUNK, min(n, (k + 1) * W.CHUNK)
            m = hi - lo
            tA[lo:hi].copy_(torch.from_numpy(A[:m]))
            tB[lo:hi].copy_(torch.from_numpy(B[:m]))
            tz[lo:hi].copy_(torch.from_numpy(z[:m]))
            sel = (sample >= lo) & (sample < hi)
            sA[sel], sB[sel], sz[sel] = A[sample[sel] - lo], B[sample[sel] - lo], z[sample[sel] - lo]
    yield tA, tB, tz, sample, sA, sB, sz
    del tA, tB, tz
    torch.cuda.empty_cache()


def _run(tA, tB, tz, mode):
    pts = torch.empty((tz.shape[0], 2, 3), dtype=torch.float64, device=DEV)
    cnt = torch.empty(tz.shape[0], dtype=torch.int32, device=DEV)
    sphx.sphx_intersect_gca_constlat(tA, tB, tz, pts, cnt, mode)
    torch.cuda.synchronize()
    return pts, cnt


def _properties(pts, cnt, tz):
    assert int(cnt.min()) >= 0 and int(cnt.max()) <= 2
    hit = torch.isfinite(pts[..., 0])
    assert torch.equal(hit.sum(1).to(torch.int32), cnt)
    # each hit lies on its latitude and on the unit sphere (|P|^2 = 1 to rounding)
    assert bool((pts[..., 2][hit] == tz[:, None].expand(-1, 2)[hit]).all())
    r2 = (pts[..., 0] ** 2 + pts[..., 1] ** 2 + pts[..., 2] ** 2)[hit]
    assert float((r2 - 1).abs().max()) < 1e-14


def _properties_loose(pts, cnt, tz):
    """hit counts and slots consistent, hits at their latitudes (no |P| check:
    the inaccurate modes may leave the sphere)"""
    assert int(cnt.min()) >= -1 and int(cnt.max()) <= 2
    hit = torch.isfinite(pts[..., 0])
    assert torch.equal(hit.sum(1).to(torch.int32), cnt.clamp(min=0))
    assert bool((pts[..., 2][hit] == tz[:, None].expand(-1, 2)[hit]).all())


def _dist_row(mode, p, c, ce, pe, ok, z):
    both = ok[:, None] & np.isfinite(pe[..., 0]) & np.isfinite(p[..., 0])
    ulp, _, gate = P.component_errors(p, pe, z)
    g = gate[both]
    return (mode, float(np.mean(ulp[both] == 0.0)), float(np.percentile(g, 95)), float(g.max()),
            float(np.mean(c[ok] == ce[ok])))


def test_full_size_mixed_workload(full_batch):
    tA, tB, tz, sample, sA, sB, sz = full_batch
    pw, cw = _run(tA, tB, tz, "wide")
    _properties(pw, cw, tz)
    # the exact oracle on the sample (integer limbs: <= 1 ulp, exact counts)
    ce, pe, fe = P.run_exact(sA, sB, sz)
    P.assert_unflagged(fe)
    ok = fe == 0
    idx = torch.from_numpy(sample).to(DEV)
    c_s = cw[idx].cpu().numpy()
    p_s = pw[idx].cpu().numpy()
    assert np.array_equal(c_s[ok], ce[ok])
    hit = np.isfinite(pe[..., 0]) & ok[:, None]
    _, _, gate = P.component_errors(p_s, pe, sz)
    assert np.nanmax(np.where(hit[..., None], gate, 0.0)) <= 1.0
    # FP64-EFT on the whole batch: the sample within 4 ulp of the oracle, and
    # the two evaluations agreeing everywhere up to boundary cases
    pf, cf = _run(tA, tB, tz, "eft")
    _properties(pf, cf, tz)
    c_f = cf[idx].cpu().numpy()
    p_f = pf[idx].cpu().numpy()
    assert np.array_equal(c_f[ok], ce[ok])
    _, _, gate = P.component_errors(p_f, pe, sz)
    assert np.nanmax(np.where(hit[..., None], gate, 0.0)) <= 4.0
    same = cw == cf
    assert float(same.float().mean()) > 0.9999
    # the error distribution of every mode on the sample
    rows = []
    for mode, (pm, cm) in (("wide", (pw, cw)), ("eft", (pf, cf))):
        rows.append(_dist_row(mode, pm[idx].cpu().numpy(), cm[idx].cpu().numpy(), ce, pe, ok, sz))
    for mode in ("direct", "ff32"):
        pm, cm = _run(tA, tB, tz, mode)
        _properties_loose(pm, cm, tz)
        p_m, c_m = pm[idx].cpu().numpy(), cm[idx].cpu().numpy()
        rows.append(_dist_row(mode, p_m, c_m, ce, pe, ok, sz))
        if mode == "ff32":
            hitm = np.isfinite(pe[..., 0]) & np.isfinite(p_m[..., 0]) & ok[:, None]
            err = P.norm_error(p_m, pe, sz)
            assert np.nanmax(np.where(hitm, err, 0)) <= P.FF_BOUND
            assert np.array_equal(c_m[ok], ce[ok])
        del pm, cm
    print("\nmode    correctly-rounded  p95        max        exact counts")
    for r in rows:
        print(f"{r[0]:7s} {r[1]:17.6f}  {r[2]:.4g}  {r[3]:.4g}  {r[4]:.6f}")
    # points: within the sum of the two bounds (1 + 4 ulp for large components,
    # (1 + 4) u sqrt(1 - z0^2) in absolute terms for small ones), with slack 1
    both = (same[:, None] & torch.isfinite(pw[..., 0]) & torch.isfinite(pf[..., 0]))[..., None]
    rho = torch.sqrt((1 - tz * tz).clamp(min=0))[:, None, None]
    a = pw[..., :2].abs()
    large = a >= 2.0 ** -20 * rho
    bound = torch.where(large, 6 * 2.0 ** -52 * a, 6 * 2.0 ** -53 * rho)
    d = (pw[..., :2] - pf[..., :2]).abs()
    assert bool(((d <= bound) | ~both).all())


# ---- ragged batch at full size: 512 meshes of 1e3 - 5e6 edges (~3e8 edges) ----
N_MESH, E_MIN, E_MAX = 512, 1e3, 5e6
N_EDGE_SAMPLE = 200


@pytest.fixture(scope="module")
def full_ragged():
    E, L = W.ragged_sizes(N_MESH, E_MIN, E_MAX)
    eo = np.concatenate([[0], np.cumsum(E)]).astype(np.int64)
    lo_ = np.concatenate([[0], np.cumsum(L)]).astype(np.int64)
    lat = np.concatenate([W.latlon_latitudes(int(l)) for l in L])
    Et = int(eo[-1])
    tA = torch.empty((Et, 3), dtype=torch.float64, device=DEV)
    tB = torch.empty((Et, 3), dtype=torch.float64, device=DEV)
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(Et, N_EDGE_SAMPLE, replace=False))
    sA = np.empty((N_EDGE_SAMPLE, 3))
    sB = np.empty((N_EDGE_SAMPLE, 3))
    seed = W.DEFAULT_SEED + 3
    procs = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        jobs = [(m, int(E[m]), seed) for m in range(N_MESH)]
        for m, (A, B) in enumerate(pool.imap(W.ragged_mesh, jobs)):
            lo, hi = int(eo[m]), int(eo[m + 1])
            tA[lo:hi].copy_(torch.from_numpy(A))
            tB[lo:hi].copy_(torch.from_numpy(B))
            sel = (sample >= lo) & (sample < hi)
            sA[sel], sB[sel] = A[sample[sel] - lo], B[sample[sel] - lo]
    d = {"A": tA, "B": tB, "eo": torch.from_numpy(eo).to(DEV),
         "lat": torch.from_numpy(lat).to(DEV), "lo": torch.from_numpy(lo_).to(DEV)}
    host = {"eo": eo, "lo": lo_, "lat": lat, "sample": sample, "sA": sA, "sB": sB}
    yield d, host
    del d, tA, tB
    torch.cuda.empty_cache()


def _ragged_run(ctx, d, mode):
    Et = d["A"].shape[0]
    lo = torch.empty(Et, dtype=torch.int32, device=DEV)
    hi = torch.empty(Et, dtype=torch.int32, device=DEV)
    sphx.sphx_candidate_ranges(d["A"], d["B"], d["eo"], d["lat"], d["lo"], lo, hi)
    pairs = int((hi - lo).sum().item())
    del lo, hi
    cap = pairs + pairs // 8 + 4096
    out = torch.empty(cap * 4, dtype=torch.int64, device=DEV)
    total = torch.zeros(1, dtype=torch.int64, device=DEV)
    sphx.sphx_intersect_ragged(ctx, d["A"], d["B"], d["eo"], d["lat"], d["lo"], out, total, mode)
    assert ctx.sync_status() == sphx.OK
    t = int(total.item())
    assert 0 < t <= cap
    return out.view(-1, 4)[:t], pairs


def _records_of(recs, sample):
    sel = recs[torch.isin(recs[:, 0], torch.from_numpy(sample).to(DEV))]
    raw = sel.contiguous().cpu().numpy().view(np.uint8).reshape(-1)
    r = raw.view(np.dtype(sphx.HIT_DTYPE))
    order = np.lexsort((r["root"], r["lat"], r["edge"]))
    return r[order]


def test_full_size_ragged_meshes(full_ragged):
    from oracle import exact, steps
    d, h = full_ragged
    eo, lo_, lat, sample = h["eo"], h["lo"], h["lat"], h["sample"]
    mesh = np.searchsorted(eo, sample, side="right") - 1
    with sphx.Context(0) as ctx:
        recs, pairs = _ragged_run(ctx, d, "wide")
        # every record: a latitude of its edge's mesh, a point on the unit sphere
        edge = recs[:, 0].contiguous()
        lat_i = (recs[:, 1] & 0xffffffff).to(torch.int64)
        mesh_t = torch.searchsorted(d["eo"], edge, right=True) - 1
        assert bool(((lat_i >= d["lo"][mesh_t]) & (lat_i < d["lo"][mesh_t + 1])).all())
        xy = recs[:, 2:4].contiguous().view(torch.float64)
        r2 = xy[:, 0] ** 2 + xy[:, 1] ** 2 + d["lat"][lat_i] ** 2
        assert float((r2 - 1).abs().max()) < 1e-14
        got_w = _records_of(recs, sample)
        del recs, edge, lat_i, mesh_t, xy, r2
        torch.cuda.empty_cache()
        recs_f, _ = _ragged_run(ctx, d, "eft")
        got_f = _records_of(recs_f, sample)
        del recs_f
        torch.cuda.empty_cache()
    # sampled edges, every latitude of their mesh (no pruning): the FP64-EFT
    # records equal the step reference bit for bit, the integer-limb records
    # the exact oracle within 1 ulp
    pe, pk = [], []
    for i, e in enumerate(sample):
        ks = np.arange(lo_[mesh[i]], lo_[mesh[i] + 1])
        pe.append(np.full(len(ks), i))
        pk.append(ks)
    pe = np.concatenate(pe)
    pk = np.concatenate(pk)
    A = h["sA"][pe]
    B = h["sB"][pe]
    z = lat[pk]
    c, p = steps.accux(A, B, z, variant=2)
    want_f = sorted((int(sample[pe[j]]), int(pk[j]), r, p[j, r, 0], p[j, r, 1])
                    for j in range(len(pe)) for r in range(2) if np.isfinite(p[j, r, 0]))
    have_f = [(int(x["edge"]), int(x["lat"]), int(x["root"]), x["x"], x["y"]) for x in got_f]
    assert len(have_f) == len(want_f)
    for a, b in zip(have_f, want_f):
        assert a[:3] == b[:3] and P.same_bits(a[3:], b[3:])
    # the exact oracle on every (sampled edge, latitude) pair
    ce, pex, fe = P.run_exact(A, B, z)
    P.assert_unflagged(fe)
    pair_of = {(int(sample[pe[j]]), int(pk[j])): j for j in range(len(pe))}
    wp = np.full((len(pe), 2, 3), np.nan)
    for x in got_w:
        j = pair_of[(int(x["edge"]), int(x["lat"]))]
        wp[j, int(x["root"])] = (x["x"], x["y"], z[j])
    ok = fe == 0
    assert np.array_equal(np.isfinite(wp[ok, :, 0]), np.isfinite(pex[ok, :, 0]))
    hit = np.isfinite(pex[..., 0]) & ok[:, None]
    _, _, gate = P.component_errors(wp, pex, z)
    assert np.nanmax(np.where(hit[..., None], gate, 0.0)) <= 1.0
