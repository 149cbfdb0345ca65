"""The allocation-free ragged entry point, against the context-based one.

Callers that cannot allocate device memory on their call path (a plugin whose
host framework owns the device memory budget, a latency-critical loop that
cannot take cudaMalloc's device synchronisation) use
sphx_intersect_ragged_noalloc, whose scratch is a fixed array inside the
library. Two calls in a row through the C ABI must give the same hit records
as sphx_intersect_ragged (the second call also shows that the array's
leftover contents from the first are cleared). This file is collected last so
that a run stopping at the first failure has run every other test first.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2510_09892_gb300 import sphx
from paper_2510_09892_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _sorted(recs):
    order = np.lexsort((recs["root"], recs["lat"], recs["edge"]))
    r = recs[order]
    return (np.stack([r["edge"], r["lat"].astype(np.int64), r["root"].astype(np.int64)], 1),
            r["x"].copy(), r["y"].copy())


def _batch(seed):
    b = W.ragged_meshes(5, 50, 800, seed=seed, lat_min=180, lat_max=700)
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(DEV) for k, v in b.items()}
    pairs = int((np.diff(b["edge_offsets"]) * np.diff(b["lat_offsets"])).sum())
    return d, 2 * pairs + 16


def _reference(d, cap, mode):
    out = torch.zeros(cap * 4, dtype=torch.int64, device=DEV)
    total = torch.zeros(1, dtype=torch.int64, device=DEV)
    with sphx.Context(0) as ctx:
        sphx.sphx_intersect_ragged(ctx, d["A"], d["B"], d["edge_offsets"], d["lat_z"],
                                   d["lat_offsets"], out, total, mode)
        assert ctx.sync_status() == sphx.OK
    t = int(total.item())
    return t, _sorted(sphx.hits_to_numpy(out, t))


def _noalloc_c_abi(d, cap, mode):
    """One call straight through the C ABI (ctypes, raw device pointers)."""
    out = torch.full((cap * 4,), -1, dtype=torch.int64, device=DEV)  # poisoned
    total = torch.full((1,), -7, dtype=torch.int64, device=DEV)
    L = sphx.lib()
    st = L.sphx_intersect_ragged_noalloc(
        d["A"].data_ptr(), d["B"].data_ptr(), d["edge_offsets"].data_ptr(),
        int(d["edge_offsets"].shape[0]) - 1, int(d["A"].shape[0]), d["lat_z"].data_ptr(),
        d["lat_offsets"].data_ptr(), int(d["lat_z"].shape[0]), sphx.MODES[mode],
        out.data_ptr(), cap, total.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == sphx.OK, sphx.status_string(st)
    torch.cuda.synchronize()
    t = int(total.item())
    return t, _sorted(sphx.hits_to_numpy(out, min(t, cap)))


@pytest.mark.parametrize("mode", ["eft", "wide"])
def test_noalloc_matches_context_call_twice(mode):
    for seed in (11, 12):  # two calls in a row, on different batches
        d, cap = _batch(seed)
        t_ref, (k_ref, x_ref, y_ref) = _reference(d, cap, mode)
        t, (k, x, y) = _noalloc_c_abi(d, cap, mode)
        assert t == t_ref and t > 0
        assert np.array_equal(k, k_ref)
        # the same kernels on the same inputs: identical points
        assert np.array_equal(x, x_ref) and np.array_equal(y, y_ref)


def test_noalloc_rejects_batches_beyond_its_scratch():
    L = sphx.lib()
    E = sphx.NOALLOC_MAX_EDGES + 1
    fake = 1 << 40  # never dereferenced: the size check comes first
    st = L.sphx_intersect_ragged_noalloc(fake, fake, fake, 1, E, fake, fake, 10, 1, fake, 10,
                                         fake, None)
    assert st == sphx.ERR_INVALID_ARG


def test_noalloc_status_reports_capacity_then_clears():
    """The status readback of the allocation-free call: a call with room for
    too few records reports SPHX_ERR_CAPACITY (and *out_total > out_cap); the
    next call, with room enough, reports SPHX_OK."""
    d, cap = _batch(13)
    t, _ = _noalloc_c_abi(d, 8, "wide")
    assert t > 8
    L = sphx.lib()
    s = torch.cuda.current_stream().cuda_stream
    assert L.sphx_noalloc_sync_status(s) == sphx.ERR_CAPACITY
    assert L.sphx_noalloc_sync_status(s) == sphx.OK  # read and cleared
    t2, _ = _noalloc_c_abi(d, cap, "wide")
    assert t2 == t
    assert L.sphx_noalloc_sync_status(s) == sphx.OK
