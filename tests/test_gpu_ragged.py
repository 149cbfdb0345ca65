"""Parity of the ragged CUDA call (sphx_intersect_ragged) with the oracle.

Expected hits come from brute force over EVERY (edge, latitude) pair of each
mesh, with no candidate pruning:
  * the step-by-step FP64 reference (oracle/accux_ref.c) on all pairs must
    give exactly the GPU's records, bit for bit (so the candidate ranges lose
    no hit and the compaction drops or duplicates none);
  * the exact oracle (oracle/ragged.py) on the sampled edges must agree on the
    hits, points within 4 ulp per component.
"""
import numpy as np
import pytest
import torch

from oracle import exact, steps
from oracle import ragged as oracle_ragged
from paper_2510_09892_gb300 import sphx
from paper_2510_09892_gb300 import workloads as W
from tests import parity as P

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def to_dev(batch):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to(DEV) for k, v in batch.items()}


def all_pairs_reference(batch, mode="eft", edges=None):
    """Brute force with the step reference: records sorted by (edge, lat, root)."""
    A, B = batch["A"], batch["B"]
    eo, lo_ = batch["edge_offsets"], batch["lat_offsets"]
    lat_z = batch["lat_z"]
    E = len(A)
    mesh_of = np.searchsorted(eo, np.arange(E), side="right") - 1
    if edges is None:
        edges = np.arange(E)
    nl = (lo_[mesh_of[edges] + 1] - lo_[mesh_of[edges]]).astype(np.int64)
    pe = np.repeat(edges, nl)
    first = np.repeat(lo_[mesh_of[edges]], nl)
    start = np.repeat(np.cumsum(nl) - nl, nl)
    pk = first + (np.arange(len(pe)) - start)
    if mode == "eft":
        c, p = steps.accux(A[pe], B[pe], lat_z[pk], variant=2)
    else:
        c, p = steps.direct(A[pe], B[pe], lat_z[pk])
    recs = []
    for r in range(2):
        h = np.isfinite(p[:, r, 0])
        recs.append(np.stack([pe[h], pk[h], np.full(h.sum(), r)], 1))
        recs[-1] = (recs[-1], p[h, r, 0], p[h, r, 1])
    key = np.concatenate([recs[0][0], recs[1][0]])
    x = np.concatenate([recs[0][1], recs[1][1]])
    y = np.concatenate([recs[0][2], recs[1][2]])
    order = np.lexsort((key[:, 2], key[:, 1], key[:, 0]))
    return key[order], x[order], y[order]


def run_ragged(ctx, d, mode="eft", cap=None, lo=None, hi=None):
    if cap is None:  # room for two hits on every (edge, latitude) pair
        eo = d["edge_offsets"].cpu().numpy()
        lo_ = d["lat_offsets"].cpu().numpy()
        cap = 16 + 2 * int((np.diff(eo) * np.diff(lo_)).sum())
    out = torch.full((cap * 4,), -1, dtype=torch.int64, device=DEV)  # 32 B records, poisoned
    total = torch.full((1,), -5, dtype=torch.int64, device=DEV)
    sphx.sphx_intersect_ragged(ctx, d["A"], d["B"], d["edge_offsets"], d["lat_z"],
                               d["lat_offsets"], out, total, mode, lo, hi)
    st = ctx.sync_status()
    t = int(total.item())
    recs = sphx.hits_to_numpy(out, min(t, cap))
    return st, t, recs


def sorted_records(recs):
    order = np.lexsort((recs["root"], recs["lat"], recs["edge"]))
    r = recs[order]
    key = np.stack([r["edge"], r["lat"].astype(np.int64), r["root"].astype(np.int64)], 1)
    return key, r["x"].copy(), r["y"].copy()


@pytest.fixture(scope="module")
def ctx():
    c = sphx.Context(0)
    yield c
    c.close()


def small_batch(seed=3):
    return W.ragged_meshes(6, 40, 600, seed=seed, lat_min=180, lat_max=500)


@pytest.mark.parametrize("compaction", [sphx.COMPACT_ATOMIC, sphx.COMPACT_ORDERED,
                                        sphx.COMPACT_FUSED])
@pytest.mark.parametrize("mode", ["eft", "direct"])
def test_small_meshes_equal_all_pairs_reference(ctx, mode, compaction):
    batch = small_batch()
    d = to_dev(batch)
    ctx.set_tuning(compaction=compaction, use_graph=1)
    st, total, recs = run_ragged(ctx, d, mode)
    assert st == sphx.OK
    key, x, y = all_pairs_reference(batch, mode)
    assert total == len(key)
    if compaction == sphx.COMPACT_ORDERED:
        got = np.stack([recs["edge"], recs["lat"].astype(np.int64),
                        recs["root"].astype(np.int64)], 1)
        gx, gy = recs["x"], recs["y"]
    else:
        got, gx, gy = sorted_records(recs)
    assert np.array_equal(got, key)
    assert P.same_bits(gx, x) and P.same_bits(gy, y)
    ctx.reset_tuning()


@pytest.mark.parametrize("compaction", [sphx.COMPACT_ATOMIC, sphx.COMPACT_FUSED])
@pytest.mark.parametrize("mode", ["eft", "wide"])
def test_small_meshes_against_exact_oracle(ctx, mode, compaction):
    batch = W.ragged_meshes(4, 20, 120, seed=9, lat_min=180, lat_max=260)
    d = to_dev(batch)
    ctx.set_tuning(compaction=compaction)
    st, total, recs = run_ragged(ctx, d, mode)
    ctx.reset_tuning()
    assert st == sphx.OK
    want, flagged, degenerate = oracle_ragged.intersect_ragged(
        batch["A"], batch["B"], batch["edge_offsets"], batch["lat_z"], batch["lat_offsets"])
    wk = {(e, k, r): (x, yy) for e, k, r, x, yy in want}
    gk, gx, gy = sorted_records(recs)
    got = {tuple(int(v) for v in gk[i]): (gx[i], gy[i]) for i in range(len(gk))}
    pairs = sum(int(eo1 - eo0) * int(lo1 - lo0) for eo0, eo1, lo0, lo1 in zip(
        batch["edge_offsets"][:-1], batch["edge_offsets"][1:],
        batch["lat_offsets"][:-1], batch["lat_offsets"][1:]))
    assert len(flagged) <= (1 - P.MIN_UNFLAGGED) * pairs
    # identical hit sets except on pairs the oracle flags as near a boundary
    diff = set(wk) ^ set(got)
    assert all((e, k) in flagged for e, k, _ in diff), sorted(diff)[:5]
    for key in set(wk) & set(got):
        e, k, r = key
        z0 = batch["lat_z"][k]
        ref = np.array([[[wk[key][0], wk[key][1], z0]] * 2])
        pts = np.array([[[got[key][0], got[key][1], z0]] * 2])
        _, _, gate = P.component_errors(pts, ref, np.array([z0]))
        assert gate.max() <= 4.0, (key, gate)


def fused_batches(kind):
    """Batches that take each path of the fused kernel: one mesh whose grid is
    staged in shared memory (cubed sphere, 721 latitudes); many small meshes,
    so that chunks of edges span mesh boundaries (grids read in global memory);
    grids larger than the staging area (3000-3500 latitudes); an empty mesh in
    the middle; a single edge."""
    if kind == "cubed":
        A, B = W.cubed_sphere_edges(12)
        return {"A": A, "B": B, "edge_offsets": np.array([0, len(A)], dtype=np.int64),
                "lat_z": W.latlon_latitudes(721), "lat_offsets": np.array([0, 721], dtype=np.int64)}
    if kind == "tiny_meshes":
        return W.ragged_meshes(40, 3, 30, seed=21, lat_min=180, lat_max=400)
    if kind == "big_grids":
        return W.ragged_meshes(3, 200, 700, seed=22, lat_min=3000, lat_max=3500)
    if kind == "empty_mesh":
        b = W.ragged_meshes(4, 100, 400, seed=23, lat_min=180, lat_max=300)
        eo, lo_ = b["edge_offsets"], b["lat_offsets"]
        b["edge_offsets"] = np.concatenate([eo[:3], eo[2:3], eo[3:]])
        b["lat_offsets"] = np.concatenate([lo_[:3], lo_[2:3], lo_[3:]])
        return b
    A, B = W.cubed_sphere_edges(2)
    return {"A": A[:1], "B": B[:1], "edge_offsets": np.array([0, 1], dtype=np.int64),
            "lat_z": W.latlon_latitudes(181), "lat_offsets": np.array([0, 181], dtype=np.int64)}


@pytest.mark.parametrize("threads,bps,ept", [(128, 4, 1), (256, 2, 1), (128, 4, 2),
                                             (256, 3, 2), (128, 8, 4), (256, 4, 4)])
@pytest.mark.parametrize("kind", ["cubed", "tiny_meshes", "big_grids", "empty_mesh", "one_edge"])
@pytest.mark.parametrize("mode", ["eft", "direct"])
def test_fused_kernel_equals_all_pairs_reference(ctx, mode, kind, threads, bps, ept):
    """The fused ragged kernel (ranges, pair queue and evaluation in one
    launch; 1, 2 or 4 edges per thread and chunk): the same records as brute
    force over every (edge, latitude) pair with the step reference, bit for
    bit, on every path of the kernel."""
    batch = fused_batches(kind)
    d = to_dev(batch)
    ctx.set_tuning(threads_per_block=threads, blocks_per_sm=bps, pairs_per_lane=ept,
                   compaction=sphx.COMPACT_FUSED, use_graph=1)
    st, total, recs = run_ragged(ctx, d, mode)
    ctx.reset_tuning()
    assert st == sphx.OK
    key, x, y = all_pairs_reference(batch, mode)
    got, gx, gy = sorted_records(recs)
    assert total == len(key) and np.array_equal(got, key)
    assert P.same_bits(gx, x) and P.same_bits(gy, y)


def test_fused_capacity_overflow_and_caller_ranges(ctx):
    """The fused kernel: a buffer with room for a third of the hits gets
    exactly its capacity of valid records, the status reports the overflow
    and *out_total the full count; caller-given ranges are used as given."""
    batch = small_batch(seed=24)
    d = to_dev(batch)
    key, x, y = all_pairs_reference(batch)
    ctx.set_tuning(compaction=sphx.COMPACT_FUSED)
    cap = len(key) // 3
    st, total, recs = run_ragged(ctx, d, "eft", cap=cap)
    assert st == sphx.ERR_CAPACITY and total == len(key) and len(recs) == cap
    kk = {tuple(r) for r in key.tolist()}
    assert all((int(r["edge"]), int(r["lat"]), int(r["root"])) in kk for r in recs)
    assert ctx.sync_status() == sphx.OK
    E = len(batch["A"])
    eo, lo_ = batch["edge_offsets"], batch["lat_offsets"]
    mesh_of = np.searchsorted(eo, np.arange(E), side="right") - 1
    full_lo = torch.from_numpy(lo_[mesh_of].astype(np.int32)).to(DEV)
    full_hi = torch.from_numpy(lo_[mesh_of + 1].astype(np.int32)).to(DEV)
    st, total, recs = run_ragged(ctx, d, "eft", lo=full_lo, hi=full_hi)
    ctx.reset_tuning()
    got, gx, gy = sorted_records(recs)
    assert st == sphx.OK and np.array_equal(got, key) and P.same_bits(gx, x)


def test_cubed_sphere_with_latlon_grid(ctx):
    A, B = W.cubed_sphere_edges(8)
    batch = {"A": A, "B": B, "edge_offsets": np.array([0, len(A)], dtype=np.int64),
             "lat_z": W.latlon_latitudes(721), "lat_offsets": np.array([0, 721], dtype=np.int64)}
    d = to_dev(batch)
    st, total, recs = run_ragged(ctx, d, "eft")
    assert st == sphx.OK
    key, x, y = all_pairs_reference(batch)
    got, gx, gy = sorted_records(recs)
    assert total == len(key) and np.array_equal(got, key)
    assert P.same_bits(gx, x) and P.same_bits(gy, y)


def test_capacity_overflow_reports_and_truncates(ctx):
    batch = small_batch(seed=4)
    d = to_dev(batch)
    key, x, y = all_pairs_reference(batch)
    cap = len(key) // 3
    ctx.set_tuning(compaction=sphx.COMPACT_ORDERED)
    st, total, recs = run_ragged(ctx, d, "eft", cap=cap)
    ctx.reset_tuning()
    assert st == sphx.ERR_CAPACITY
    assert total == len(key)
    assert len(recs) == cap
    got = np.stack([recs["edge"], recs["lat"].astype(np.int64), recs["root"].astype(np.int64)], 1)
    assert np.array_equal(got, key[:cap])
    # the status word is cleared once read
    assert ctx.sync_status() == sphx.OK


def test_caller_ranges_and_candidate_ranges(ctx):
    batch = small_batch(seed=5)
    d = to_dev(batch)
    E = len(batch["A"])
    eo, lo_ = batch["edge_offsets"], batch["lat_offsets"]
    mesh_of = np.searchsorted(eo, np.arange(E), side="right") - 1
    full_lo = torch.from_numpy(lo_[mesh_of].astype(np.int32)).to(DEV)
    full_hi = torch.from_numpy(lo_[mesh_of + 1].astype(np.int32)).to(DEV)
    st, total, recs = run_ragged(ctx, d, "eft", lo=full_lo, hi=full_hi)
    assert st == sphx.OK
    key, x, y = all_pairs_reference(batch)
    got, gx, gy = sorted_records(recs)
    assert np.array_equal(got, key) and P.same_bits(gx, x)
    # the computed ranges cover every hit and are far narrower than the grids
    lo = torch.empty(E, dtype=torch.int32, device=DEV)
    hi = torch.empty(E, dtype=torch.int32, device=DEV)
    sphx.sphx_candidate_ranges(d["A"], d["B"], d["edge_offsets"], d["lat_z"], d["lat_offsets"],
                               lo, hi)
    lo, hi = lo.cpu().numpy(), hi.cpu().numpy()
    e, k = key[:, 0], key[:, 1]
    assert ((lo[e] <= k) & (k < hi[e])).all()
    assert ((lo >= lo_[mesh_of]) & (hi <= lo_[mesh_of + 1])).all()
    assert (hi - lo).sum() < 0.5 * (lo_[mesh_of + 1] - lo_[mesh_of]).sum()


def test_empty_batches_and_empty_meshes(ctx):
    batch = small_batch(seed=6)
    # insert an empty mesh in the middle
    eo = batch["edge_offsets"]
    batch["edge_offsets"] = np.concatenate([eo[:3], eo[2:3], eo[3:]])
    lo_ = batch["lat_offsets"]
    batch["lat_offsets"] = np.concatenate([lo_[:3], lo_[2:3] + 0, lo_[3:]])
    d = to_dev(batch)
    st, total, recs = run_ragged(ctx, d, "eft")
    assert st == sphx.OK
    key, _, _ = all_pairs_reference(batch)
    assert total == len(key)
    # E = 0
    e0 = {"A": torch.zeros((0, 3), dtype=torch.float64, device=DEV),
          "B": torch.zeros((0, 3), dtype=torch.float64, device=DEV),
          "edge_offsets": torch.zeros(2, dtype=torch.int64, device=DEV),
          "lat_z": d["lat_z"], "lat_offsets": d["lat_offsets"][:2].clone()}
    e0["lat_offsets"][0] = 0
    st, total, recs = run_ragged(ctx, e0, "eft", cap=16)
    assert st == sphx.OK and total == 0


def test_graph_replay_sees_new_inputs(ctx):
    b1 = small_batch(seed=7)
    d = to_dev(b1)
    st, t1, _ = run_ragged(ctx, d, "eft")
    # overwrite the endpoints in place (same pointers -> the cached graph replays)
    b2 = dict(b1)
    b2["B"] = np.ascontiguousarray(b1["A"][::-1])
    b2["A"] = np.ascontiguousarray(b1["B"][::-1])
    d["A"].copy_(torch.from_numpy(b2["A"]))
    d["B"].copy_(torch.from_numpy(b2["B"]))
    st, t2, recs = run_ragged(ctx, d, "eft")
    key, x, y = all_pairs_reference(b2)
    got, gx, gy = sorted_records(recs)
    assert st == sphx.OK and np.array_equal(got, key) and P.same_bits(gx, x)


def test_autotune_then_correct(ctx):
    batch = small_batch(seed=8)
    d = to_dev(batch)
    # a buffer too small for the batch: the trials overflow it, and the
    # autotuner must not leave that status behind for the next call
    out = torch.empty(4 * 8, dtype=torch.int64, device=DEV)
    total = torch.empty(1, dtype=torch.int64, device=DEV)
    ms = sphx.sphx_autotune_ragged(ctx, d["A"], d["B"], d["edge_offsets"], d["lat_z"],
                                   d["lat_offsets"], out, total, "eft")
    assert ms > 0
    t = ctx.get_tuning()
    assert t["threads_per_block"] in (128, 256) and t["use_graph"] == 1
    assert ctx.sync_status() == sphx.OK
    st, total, recs = run_ragged(ctx, d, "eft")
    key, x, y = all_pairs_reference(batch)
    got, gx, gy = sorted_records(recs)
    assert st == sphx.OK and np.array_equal(got, key) and P.same_bits(gx, x)
    ctx.reset_tuning()


def test_full_size_cubed_sphere_sampled(ctx):
    """The regridding workload at full size (N = 1024, 12 595 200 edges, 721
    latitudes) in the benchmark's launch shape: the records of 3000 seeded
    sampled edges equal the all-pairs step reference bit for bit, and every
    record is a valid pair whose point lies on the unit sphere."""
    A, B = W.cubed_sphere_edges(1024)
    batch = {"A": A, "B": B, "edge_offsets": np.array([0, len(A)], dtype=np.int64),
             "lat_z": W.latlon_latitudes(721), "lat_offsets": np.array([0, 721], dtype=np.int64)}
    d = to_dev(batch)
    cap = 4 * len(A)
    st, total, recs = run_ragged(ctx, d, "eft", cap=cap)
    assert st == sphx.OK
    sample = np.sort(np.random.default_rng(1).choice(len(A), 3000, replace=False))
    key, x, y = all_pairs_reference(batch, edges=sample)
    sel = np.isin(recs["edge"], sample)
    got, gx, gy = sorted_records(recs[sel])
    assert np.array_equal(got, key)
    assert P.same_bits(gx, x) and P.same_bits(gy, y)
    # every record is a valid pair with a point on its latitude's circle
    assert (recs["lat"] >= 0).all() and (recs["lat"] < 721).all()
    z0 = batch["lat_z"][recs["lat"]]
    r2 = recs["x"] ** 2 + recs["y"] ** 2 + z0 ** 2
    assert np.abs(r2 - 1).max() < 1e-14


def test_injected_lookback_stall_times_out_and_context_recovers(monkeypatch):
    """Failure injection on the host side: with SPHX_FAULT=lookback the first
    chunk of the ordered compaction never publishes its prefix, so the next
    chunk's look-back waits on a flag that nothing sets. The wait is bounded:
    the call ends, sync_status reports ERR_TIMEOUT, and the same context then
    gives the exact records once the fault is lifted."""
    batch = W.ragged_meshes(2, 40, 80, seed=12, lat_min=180, lat_max=260)
    d = to_dev(batch)
    key, x, y = all_pairs_reference(batch)
    assert len(key) > 64  # more than one chunk of 32 pairs
    with sphx.Context(0) as c:
        c.set_tuning(compaction=sphx.COMPACT_ORDERED, use_graph=0)
        monkeypatch.setenv("SPHX_FAULT", "lookback")
        st, _, _ = run_ragged(c, d, "eft")
        assert st == sphx.ERR_TIMEOUT
        monkeypatch.delenv("SPHX_FAULT")
        assert c.sync_status() == sphx.OK  # the status word was cleared
        st, total, recs = run_ragged(c, d, "eft")
        assert st == sphx.OK and total == len(key)
        got = np.stack([recs["edge"], recs["lat"].astype(np.int64),
                        recs["root"].astype(np.int64)], 1)
        assert np.array_equal(got, key) and P.same_bits(recs["x"], x)


def test_injected_scratch_allocation_failure(monkeypatch):
    """SPHX_FAULT=alloc makes the scratch allocation of a fresh context fail:
    the call returns ERR_NOMEM before any launch, and the context works once
    the fault is lifted."""
    batch = small_batch(seed=13)
    d = to_dev(batch)
    with sphx.Context(0) as c:
        monkeypatch.setenv("SPHX_FAULT", "alloc")
        with pytest.raises(sphx.SphxError) as ei:
            run_ragged(c, d, "eft")
        assert ei.value.status == sphx.ERR_NOMEM
        monkeypatch.delenv("SPHX_FAULT")
        st, total, recs = run_ragged(c, d, "eft")
        key, x, y = all_pairs_reference(batch)
        got, gx, gy = sorted_records(recs)
        assert st == sphx.OK and np.array_equal(got, key) and P.same_bits(gx, x)


def test_tuning_cache_reused_by_a_second_context():
    """The autotuners' results are kept per (device, call, mode, size class):
    a second context autotuning the same batch takes the shape from the cache
    without a sweep, and so does the dense autotuner on a second call."""
    sphx.tuning_cache_clear()
    batch = small_batch(seed=25)
    d = to_dev(batch)
    out = torch.empty(4 * 200_000, dtype=torch.int64, device=DEV)
    total = torch.empty(1, dtype=torch.int64, device=DEV)
    with sphx.Context(0) as c1:
        ms1 = sphx.sphx_autotune_ragged(c1, d["A"], d["B"], d["edge_offsets"], d["lat_z"],
                                        d["lat_offsets"], out, total, "wide")
        t1 = c1.get_tuning()
    assert sphx.tuning_cache_stats() == (0, 1)
    with sphx.Context(0) as c2:
        ms2 = sphx.sphx_autotune_ragged(c2, d["A"], d["B"], d["edge_offsets"], d["lat_z"],
                                        d["lat_offsets"], out, total, "wide")
        assert c2.get_tuning() == t1 and ms2 == ms1
        st, n, recs = run_ragged(c2, d, "wide")
        assert st == sphx.OK and n > 0
    assert sphx.tuning_cache_stats() == (1, 1)
    A, B, z = W.uniform_arcs(300_000, seed=26)
    tA, tB, tz = (torch.from_numpy(v).to(DEV) for v in (A, B, z))
    pts = torch.empty((len(z), 2, 3), dtype=torch.float64, device=DEV)
    cnt = torch.empty(len(z), dtype=torch.int32, device=DEV)
    sphx.sphx_autotune_dense(tA, tB, tz, pts, cnt, "wide")
    sphx.sphx_autotune_dense(tA, tB, tz, pts, cnt, "wide")
    assert sphx.tuning_cache_stats() == (2, 2)
    # the dense call with the tuned grid gives the same results as one wave
    sphx.sphx_intersect_gca_constlat(tA, tB, tz, pts, cnt, "wide")
    p1, c1_ = pts.cpu().numpy(), cnt.cpu().numpy()
    sphx.tuning_cache_clear()
    sphx.sphx_intersect_gca_constlat(tA, tB, tz, pts, cnt, "wide")
    assert np.array_equal(c1_, cnt.cpu().numpy()) and P.same_bits(p1, pts.cpu().numpy())


_CACHE_CHILD = r"""
import json, sys, torch
sys.path.insert(0, sys.argv[1])
from paper_2510_09892_gb300 import sphx, workloads as W
b = W.ragged_meshes(6, 40, 600, seed=27, lat_min=180, lat_max=500)
dev = torch.device("cuda:0")
d = {k: torch.from_numpy(v).to(dev) for k, v in b.items()}
out = torch.empty(4 * 200000, dtype=torch.int64, device=dev)
total = torch.empty(1, dtype=torch.int64, device=dev)
with sphx.Context(0) as c:
    ms = sphx.sphx_autotune_ragged(c, d["A"], d["B"], d["edge_offsets"], d["lat_z"],
                                   d["lat_offsets"], out, total, "eft")
    print(json.dumps({"stats": sphx.tuning_cache_stats(), "tuning": c.get_tuning(), "ms": ms}))
"""


def test_tuning_cache_persists_across_processes(tmp_path):
    """With SPHX_TUNE_CACHE naming a file, the first process sweeps and writes
    the entry; a second process reads it and tunes without a sweep."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, SPHX_TUNE_CACHE=str(tmp_path / "tune.json"))
    runs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", _CACHE_CHILD, root], env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        runs.append(json.loads(r.stdout.strip().splitlines()[-1]))
    assert runs[0]["stats"] == [0, 1] and runs[1]["stats"] == [1, 0]
    assert runs[0]["tuning"] == runs[1]["tuning"]
    text = (tmp_path / "tune.json").read_text()
    assert "|ragged|mode=1|" in text and json.loads(text)
