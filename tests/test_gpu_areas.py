"""Parity of the band-area CUDA calls (sphx_band_ranges / sphx_band_areas /
sphx_zonal_sums) with the band-area oracle (oracle/areas.py).

Every (cell, band) entry is compared with the oracle's, within
32 u (sum_arcs |dlambda| + the cell's height range) (u = 2^-53): the GPU's
boundary integral sums terms of the size of each arc piece's longitude span
times its height, and each FP64 crossing point is off the exact one by a
unit of rounding along its latitude, which moves the piece's area by that
times the piece's height; so the absolute error scales with the cell's
longitude perimeter and height, not its area.
Bands outside a cell's range must be empty in the oracle too. At the bench's
size (cubed sphere N = 1024, 721 latitudes) every band's total must be
2 pi dz (Archimedes), every cell's bands must add up to its area, and
sampled cells must match the oracle.
"""
import math

import numpy as np
import pytest
import torch

from oracle import areas as OA
from paper_2510_09892_gb300 import sphx
from paper_2510_09892_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
U = 2.0 ** -53
TWO_PI = 2 * math.pi


@pytest.fixture(scope="module")
def ctx():
    c = sphx.Context(0)
    yield c
    c.close()


def _sph(lon_deg, lat_deg):
    lo, la = math.radians(lon_deg), math.radians(lat_deg)
    return (math.cos(la) * math.cos(lo), math.cos(la) * math.sin(lo), math.sin(la))


def special_cells():
    """Octant (an arc on the equator, a pole node), a pole-to-pole lune, caps
    around both poles, a quadrilateral whose nodes lie exactly on 10-degree
    latitudes, and a thin sliver across the equator."""
    z10 = [math.sin(math.radians(d)) for d in (20, 40)]
    quad = []
    for lon, z in ((15, z10[0]), (55, z10[0]), (55, z10[1]), (15, z10[1])):
        r = math.sqrt(1 - z * z)
        quad.append((r * math.cos(math.radians(lon)), r * math.sin(math.radians(lon)), z))
    cap_n = [_sph(360.0 * i / 5 + 7.0, 70) for i in range(5)]
    cap_s = [(x, y, -z) for (x, y, z) in reversed([_sph(360.0 * i / 7, 80) for i in range(7)])]
    return [
        [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)],
        [(0.0, 0.0, 1.0), _sph(10, 0), (0.0, 0.0, -1.0), _sph(47, 0)],
        cap_n, cap_s, quad,
        [_sph(100, -1e-3), _sph(100.000001, -1e-3), _sph(100.000001, 2e-3), _sph(100, 2e-3)],
    ]


def to_mesh(cells):
    k = [len(c) for c in cells]
    nodes = np.array([v for c in cells for v in c], dtype=np.float64)
    off = np.concatenate([[0], np.cumsum(k)]).astype(np.int64)
    return nodes, off, np.arange(len(nodes), dtype=np.int32)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def gpu_dense(ctx, nodes, off, fn, lat, mode):
    """GPU band areas as a dense (cells, bands) array (0 outside each range)."""
    lo, hi, ao, A = sphx.band_areas(ctx, dev(nodes), dev(off), dev(fn), dev(lat), mode)
    assert ctx.sync_status() == sphx.OK
    lo, hi, ao, A = (t.cpu().numpy() for t in (lo, hi, ao, A))
    F, nb = len(off) - 1, len(lat) - 1
    D = np.zeros((F, nb))
    for f in range(F):
        D[f, lo[f]:hi[f]] = A[ao[f]:ao[f + 1]]
    return D, lo, hi


def lon_perimeter(cells):
    """sum of |principal longitude step| between consecutive nodes off the
    poles (a pole node's arcs are meridians: the step happens across it)"""
    out = []
    for c in cells:
        v = np.asarray(c)
        v = v[np.hypot(v[:, 0], v[:, 1]) > 0]
        w = np.roll(v, -1, axis=0)
        d = np.arctan2(v[:, 0] * w[:, 1] - v[:, 1] * w[:, 0], v[:, 0] * w[:, 0] + v[:, 1] * w[:, 1])
        out.append(np.abs(d).sum())
    return np.array(out)


def error_scale(cells):
    """longitude perimeter + height range of each cell (the error's scale)"""
    zr = np.array([np.ptp(OA.breakpoints(c)) for c in cells])
    return lon_perimeter(cells) + zr


def check_against_oracle(ctx, cells, lat, modes=("wide", "eft"), factor=32.0):
    nodes, off, fn = to_mesh(cells)
    ref = np.array(OA.band_areas_batch(cells, lat, processes=8))
    tol = factor * U * error_scale(cells)
    for mode in modes:
        D, lo, hi = gpu_dense(ctx, nodes, off, fn, lat, mode)
        err = np.abs(D - ref)
        bad = err > tol[:, None]
        assert not bad.any(), (mode, np.argwhere(bad)[:5], (err / tol[:, None]).max())
        # bands outside each cell's range hold nothing in the oracle either
        for f in range(len(cells)):
            outside = np.ones(len(lat) - 1, bool)
            outside[lo[f]:hi[f]] = False
            assert np.all(ref[f, outside] <= tol[f]), (mode, f)


def test_random_polygons_vs_oracle(ctx):
    nodes, off, fn = W.polygon_cells(160, seed=31, radius=(1e-4, 0.5))
    cells = W.cells_as_lists(nodes, off, fn)
    check_against_oracle(ctx, cells, W.latlon_latitudes(91))


def test_random_latitudes_vs_oracle(ctx):
    nodes, off, fn = W.polygon_cells(60, seed=32, radius=(1e-3, 0.8))
    cells = W.cells_as_lists(nodes, off, fn)
    lat = np.sort(np.random.default_rng(5).uniform(-0.99, 0.99, 40))
    check_against_oracle(ctx, cells, lat, modes=("wide", "eft", "eft_printed"))


@pytest.mark.parametrize("N", [3, 4])
def test_cubed_sphere_vs_oracle_and_partition(ctx, N):
    """Odd N: the poles lie inside cells; even N: the poles are nodes."""
    nodes, off, fn = W.cubed_sphere_cells(N)
    cells = W.cells_as_lists(nodes, off, fn)
    lat = W.latlon_latitudes(19)
    check_against_oracle(ctx, cells, lat)
    D, _, _ = gpu_dense(ctx, nodes, off, fn, lat, "wide")
    np.testing.assert_allclose(D.sum(axis=0), TWO_PI * np.diff(lat), rtol=0, atol=1e-14)


def test_scaled_nodes_vs_oracle(ctx):
    """Nodes are directions of any nonzero length: the same polygons with every
    node scaled by 10^-3 .. 10^3 (the normalisation's reciprocal-square-root
    path) and by 1 + up to 2^-22 (its series path) match the oracle, which
    normalises the nodes itself."""
    nodes, off, fn = W.polygon_cells(60, seed=34, radius=(1e-3, 0.5))
    rng = np.random.default_rng(35)
    half = len(nodes) // 2
    scale = np.concatenate([10.0 ** rng.uniform(-3, 3, half),
                            1 + rng.uniform(-2.0 ** -22, 2.0 ** -22, len(nodes) - half)])
    nodes = np.ascontiguousarray(nodes * scale[:, None])
    cells = W.cells_as_lists(nodes, off, fn)
    check_against_oracle(ctx, cells, W.latlon_latitudes(91))


def test_special_cells_vs_oracle(ctx):
    cells = special_cells()
    check_against_oracle(ctx, cells, W.latlon_latitudes(19))
    lat = [-1.0, -0.999, -0.95, -0.2, 0.0, 1e-4, 0.3, 0.93, 0.99, 1.0]
    check_against_oracle(ctx, cells, lat)


def test_other_modes_close(ctx):
    """Direct FP64 and float-float: crossings lose accuracy near tangency, the
    areas only slightly (looser bound)."""
    nodes, off, fn = W.polygon_cells(60, seed=33, radius=(1e-3, 0.5))
    cells = W.cells_as_lists(nodes, off, fn)
    check_against_oracle(ctx, cells, W.latlon_latitudes(46), modes=("direct", "ff32"),
                         factor=2.0 ** 20)


def test_zonal_sums_exact_and_reproducible(ctx):
    nodes, off, fn = W.cubed_sphere_cells(24)
    lat = W.latlon_latitudes(73)
    lo, hi, ao, A = sphx.band_areas(ctx, dev(nodes), dev(off), dev(fn), dev(lat), "wide")
    F, nb = len(off) - 1, len(lat) - 1
    field = np.random.default_rng(2).standard_normal(F)
    fd = dev(field)
    outs = []
    for _ in range(2):
        fa = torch.empty(nb, dtype=torch.float64, device=DEV)
        aa = torch.empty(nb, dtype=torch.float64, device=DEV)
        sphx.sphx_zonal_sums(ctx, lo, hi, ao, A, fd, len(lat), fa, aa)
        assert ctx.sync_status() == sphx.OK
        outs.append((fa.cpu().numpy(), aa.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    lo, hi, ao, A = (t.cpu().numpy() for t in (lo, hi, ao, A))
    terms_fa = [[] for _ in range(nb)]
    terms_a = [[] for _ in range(nb)]
    for f in range(F):
        for j, k in enumerate(range(lo[f], hi[f])):
            terms_fa[k].append(float(field[f] * A[ao[f] + j]))
            terms_a[k].append(float(A[ao[f] + j]))
    for k in range(nb):
        n = len(terms_a[k])
        for got, terms in ((outs[0][0][k], terms_fa[k]), (outs[0][1][k], terms_a[k])):
            exact = math.fsum(terms)
            assert abs(got - exact) <= 2 * U * abs(exact) + n * 2.0 ** -80, (k, got, exact)
    np.testing.assert_allclose(outs[0][1], TWO_PI * np.diff(lat), rtol=0, atol=1e-13)


def test_invalid_node_index_and_capacity(ctx):
    cells = special_cells()
    nodes, off, fn = to_mesh(cells)
    fn_bad = fn.copy()
    fn_bad[5] = len(nodes) + 7
    lat = W.latlon_latitudes(19)
    F = len(off) - 1
    lo = torch.empty(F, dtype=torch.int32, device=DEV)
    hi = torch.empty(F, dtype=torch.int32, device=DEV)
    ao = torch.empty(F + 1, dtype=torch.int64, device=DEV)
    sphx.sphx_band_ranges(ctx, dev(nodes), dev(off), dev(fn_bad), dev(lat), lo, hi, ao)
    assert ctx.sync_status() == sphx.ERR_INVALID_ARG
    cell_of_5 = int(np.searchsorted(off, 5, side="right") - 1)
    assert int(lo[cell_of_5]) == int(hi[cell_of_5])
    # capacity: room for one entry only
    sphx.sphx_band_ranges(ctx, dev(nodes), dev(off), dev(fn), dev(lat), lo, hi, ao)
    assert ctx.sync_status() == sphx.OK
    assert int(ao[-1]) > 1
    small = torch.zeros(1, dtype=torch.float64, device=DEV)
    sphx.sphx_band_areas(ctx, dev(nodes), dev(off), dev(fn), dev(lat), lo, hi, ao, small)
    assert ctx.sync_status() == sphx.ERR_CAPACITY


def test_empty_mesh(ctx):
    nodes = torch.zeros((1, 3), dtype=torch.float64, device=DEV)
    off = torch.zeros(1, dtype=torch.int64, device=DEV)
    fn = torch.zeros(1, dtype=torch.int32, device=DEV)
    lat = dev(W.latlon_latitudes(5))
    lo = torch.empty(0, dtype=torch.int32, device=DEV)
    hi = torch.empty(0, dtype=torch.int32, device=DEV)
    ao = torch.full((1,), 7, dtype=torch.int64, device=DEV)
    sphx.sphx_band_ranges(ctx, nodes, off, fn, lat, lo, hi, ao)
    assert int(ao[0]) == 0 and ctx.sync_status() == sphx.OK


def test_full_size_cubed_sphere(ctx):
    """The bench's workload: N = 1024 (6,291,456 cells), 721 latitudes."""
    N = 1024
    nodes, off, fn = W.cubed_sphere_cells(N)
    lat = W.latlon_latitudes(721)
    dn, do, df, dl = dev(nodes), dev(off), dev(fn), dev(lat)
    lo, hi, ao, A = sphx.band_areas(ctx, dn, do, df, dl, "wide")
    assert ctx.sync_status() == sphx.OK
    F, nb = len(off) - 1, len(lat) - 1
    ones = torch.ones(F, dtype=torch.float64, device=DEV)
    fa = torch.empty(nb, dtype=torch.float64, device=DEV)
    aa = torch.empty(nb, dtype=torch.float64, device=DEV)
    sphx.sphx_zonal_sums(ctx, lo, hi, ao, A, ones, len(lat), fa, aa)
    assert ctx.sync_status() == sphx.OK
    np.testing.assert_allclose(aa.cpu().numpy(), TWO_PI * np.diff(lat), rtol=0, atol=1e-12)
    assert torch.equal(fa, aa)
    # every cell's bands add up to its area (Van Oosterom-Strackee on the two
    # triangles of the quadrilateral, in FP64 with difference vectors)
    Ah = A.cpu().numpy()
    aoh = ao.cpu().numpy()
    per_cell = np.add.reduceat(Ah, aoh[:-1]) if len(Ah) else np.zeros(F)
    q = nodes[fn.reshape(-1, 4)]

    def excess(a, b, c):
        num = np.einsum("ij,ij->i", a, np.cross(b - a, c - a))
        den = 1 + np.einsum("ij,ij->i", a, b) + np.einsum("ij,ij->i", b, c) + \
            np.einsum("ij,ij->i", c, a)
        return 2 * np.arctan2(num, den)

    girard = excess(q[:, 0], q[:, 1], q[:, 2]) + excess(q[:, 0], q[:, 2], q[:, 3])
    np.testing.assert_allclose(per_cell, girard, rtol=1e-9)
    # sampled cells (including the four around each pole) against the oracle
    rng = np.random.default_rng(17)
    pole_nodes = [int(np.argmax(nodes[:, 2])), int(np.argmin(nodes[:, 2]))]
    around = np.nonzero(np.isin(fn.reshape(-1, 4), pole_nodes).any(axis=1))[0]
    sample = np.unique(np.concatenate([rng.choice(F, 40, replace=False), around]))
    cells = W.cells_as_lists(nodes, off, fn, sample)
    ref = np.array(OA.band_areas_batch(cells, lat, processes=8))
    loh, hih = lo.cpu().numpy(), hi.cpu().numpy()
    tol = 32 * U * error_scale(cells)
    for i, f in enumerate(sample):
        got = np.zeros(nb)
        got[loh[f]:hih[f]] = Ah[aoh[f]:aoh[f + 1]]
        assert np.abs(got - ref[i]).max() <= tol[i], (f, np.abs(got - ref[i]).max(), tol[i])


def test_many_latitudes_global_paths(ctx):
    """More latitudes than the kernels stage in shared memory: the area kernel
    reads them (and computes their radii) from global memory, and the zonal
    sums accumulate in global memory (3500 bands)."""
    nodes, off, fn = W.polygon_cells(40, seed=34, radius=(1e-3, 0.3))
    cells = W.cells_as_lists(nodes, off, fn)
    lat = np.concatenate([[-1.0], np.sort(np.random.default_rng(8).uniform(-1, 1, 3499)), [1.0]])
    check_against_oracle(ctx, cells, lat, modes=("wide",))
    lo, hi, ao, A = sphx.band_areas(ctx, dev(nodes), dev(off), dev(fn), dev(lat), "wide")
    F, nb = len(off) - 1, len(lat) - 1
    field = dev(np.arange(F, dtype=np.float64))
    fa = torch.empty(nb, dtype=torch.float64, device=DEV)
    aa = torch.empty(nb, dtype=torch.float64, device=DEV)
    sphx.sphx_zonal_sums(ctx, lo, hi, ao, A, field, len(lat), fa, aa)
    assert ctx.sync_status() == sphx.OK
    lo, hi, ao, A = (t.cpu().numpy() for t in (lo, hi, ao, A))
    want_a = np.zeros(nb)
    want_fa = np.zeros(nb)
    for f in range(F):
        want_a[lo[f]:hi[f]] += A[ao[f]:ao[f + 1]]
        want_fa[lo[f]:hi[f]] += f * A[ao[f]:ao[f + 1]]
    np.testing.assert_allclose(aa.cpu().numpy(), want_a, rtol=1e-14, atol=1e-300)
    np.testing.assert_allclose(fa.cpu().numpy(), want_fa, rtol=1e-14, atol=1e-300)


def test_one_call_zonal_sums(ctx):
    """sphx.zonal_sums (ranges + areas + sums in one call) equals the three
    calls made by hand, bit for bit, and its band totals are 2 pi dz."""
    nodes, off, fn = W.cubed_sphere_cells(16)
    lat = W.latlon_latitudes(37)
    field = dev(np.random.default_rng(9).standard_normal(len(off) - 1))
    fa, aa = sphx.zonal_sums(ctx, dev(nodes), dev(off), dev(fn), dev(lat), field)
    lo, hi, ao, A = sphx.band_areas(ctx, dev(nodes), dev(off), dev(fn), dev(lat), "wide")
    fa2 = torch.empty_like(fa)
    aa2 = torch.empty_like(aa)
    sphx.sphx_zonal_sums(ctx, lo, hi, ao, A, field, len(lat), fa2, aa2)
    assert ctx.sync_status() == sphx.OK
    assert torch.equal(fa, fa2) and torch.equal(aa, aa2)
    np.testing.assert_allclose(aa.cpu().numpy(), TWO_PI * np.diff(lat), rtol=0, atol=1e-14)


def test_big_cells_in_one_band(ctx):
    """Cells of up to ~70 degrees radius inside one wide band: the one-band list
    takes them, but with nodes more than 60 degrees from node 0 the triangle
    fan passes them on to the boundary integral; cells that stick out of the
    band stay with the boundary integral from the start."""
    nodes, off, fn = W.polygon_cells(60, seed=35, radius=(0.3, 1.2), star=0.1)
    cells = W.cells_as_lists(nodes, off, fn)
    lat = np.array([-1.0, -0.999, 0.999, 1.0])
    check_against_oracle(ctx, cells, lat)
    lat = np.array([-1.0, -0.95, -0.3, 0.2, 0.97, 1.0])
    check_against_oracle(ctx, cells, lat)


def test_cells_with_many_nodes(ctx):
    """Polygons of 17-24 nodes: more than the two-band path keeps, so cells cut
    by one latitude go to the boundary integral; one-band cells still take the
    triangle fan."""
    nodes, off, fn = W.polygon_cells(80, seed=36, radius=(2e-3, 0.05), kmin=17, kmax=24)
    cells = W.cells_as_lists(nodes, off, fn)
    check_against_oracle(ctx, cells, W.latlon_latitudes(361))


def test_both_crossings_on_one_arc(ctx):
    """A latitude just above a quadrilateral's top corners: the top arc (a great
    circle between two points at one latitude) bulges poleward across it and
    back, so one arc holds both crossings (rising first); the mirror image in
    the south has them on its bottom arc, falling first."""
    north = [_sph(20, 30), _sph(50, 30), _sph(50, 31), _sph(20, 31)]
    south = [(x, y, -z) for (x, y, z) in reversed(north)]
    zt = math.sin(math.radians(31))
    apex = max(OA.breakpoints([_sph(50, 31), _sph(20, 31)]))
    assert apex > zt
    zj = 0.5 * (zt + apex)
    lat = [-1.0, 0.3, 0.49, zj, apex + 0.01, 0.9, 1.0]
    check_against_oracle(ctx, [north], lat)
    check_against_oracle(ctx, [south], [-z for z in reversed(lat)])
