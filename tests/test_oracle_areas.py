"""Pins of the band-area oracle (oracle/areas.py) against what geometry fixes.

* Archimedes: a complete mesh covers every band exactly once, so the cells'
  areas in band k add up to 2 pi (z_{k+1} - z_k) (cubed spheres with the poles
  as nodes and inside cells).
* Each cell's band areas add up to its area by the Van Oosterom-Strackee
  triangle formula (exact rational numerator and denominator).
* Closed forms: the octant and a lune (W(z) constant), a quadrilateral between
  two meridians (W = the meridians' separation between its top and bottom
  arcs), a regular polygon around a pole (Todhunter's isosceles-triangle
  excess, and W = 2 pi above its boundary).
* Symmetry: mirroring z -> -z (with the vertex order reversed to keep the
  orientation) maps band k to band L - 2 - k.
* Quadrature: more nodes change nothing beyond rounding.
"""
import math

import numpy as np
import pytest

from oracle import areas
from paper_2510_09892_gb300 import workloads as W

TWO_PI = 2 * math.pi


def _sph(lon_deg, lat_deg):
    lo, la = math.radians(lon_deg), math.radians(lat_deg)
    return (math.cos(la) * math.cos(lo), math.cos(la) * math.sin(lo), math.sin(la))


@pytest.mark.parametrize("N", [3, 4])
def test_partition_of_the_sphere(N):
    """Every band's total over a complete cubed sphere is 2 pi dz (Archimedes)."""
    nodes, off, fn = W.cubed_sphere_cells(N)
    cells = W.cells_as_lists(nodes, off, fn)
    if N == 3:
        assert sorted({areas.winding(c) for c in cells}) == [-1, 0, 1]  # polar cells
    lat = np.concatenate([[-1.0], np.sort(np.random.default_rng(N).uniform(-1, 1, 5)), [1.0]])
    A = np.array(areas.band_areas_batch(cells, lat))
    np.testing.assert_allclose(A.sum(axis=0), TWO_PI * np.diff(lat), rtol=0, atol=1e-14)
    assert (A >= -1e-16).all()


def test_partition_with_latitudes_inside():
    """Latitudes that stop short of the poles leave the polar caps out."""
    nodes, off, fn = W.cubed_sphere_cells(3)
    cells = W.cells_as_lists(nodes, off, fn)
    lat = np.array([-0.97, -0.5, 0.0, 0.31, 0.999])
    A = np.array(areas.band_areas_batch(cells, lat))
    np.testing.assert_allclose(A.sum(axis=0), TWO_PI * np.diff(lat), rtol=0, atol=1e-14)


def test_bands_add_up_to_the_cell_area():
    nodes, off, fn = W.polygon_cells(24, radius=(1e-3, 0.5))
    cells = W.cells_as_lists(nodes, off, fn)
    lat = W.latlon_latitudes(91)
    A = np.array(areas.band_areas_batch(cells, lat))
    ca = np.array([areas.cell_area(c) for c in cells])
    assert (ca > 0).all()
    np.testing.assert_allclose(A.sum(axis=1), ca, rtol=2e-14, atol=0)


def test_octant():
    """The octant x, y, z >= 0: W(z) = pi / 2 on [0, 1]; one arc is on the equator
    and one vertex is the pole."""
    cell = [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)]
    lat = [-1.0, -0.2, 0.0, 0.1, 0.5, 0.75, 1.0]
    A = areas.band_areas(cell, lat)
    expect = [0.5 * math.pi * max(0.0, min(b, 1.0) - max(a, 0.0)) for a, b in zip(lat, lat[1:])]
    np.testing.assert_allclose(A, expect, rtol=1e-15, atol=1e-16)
    assert areas.cell_area(cell) == pytest.approx(0.5 * math.pi, rel=1e-15)


def test_lune():
    """Between the meridians 10 and 47 degrees from pole to pole: W = 37 degrees."""
    cell = [(0.0, 0.0, 1.0), _sph(10, 0), (0.0, 0.0, -1.0), _sph(47, 0)]
    lat = W.latlon_latitudes(13)
    A = areas.band_areas(cell, lat)
    np.testing.assert_allclose(A, math.radians(37) * np.diff(lat), rtol=1e-14, atol=0)


def test_quadrilateral_between_meridians():
    """Vertices at (lon, lat) = (20, 30), (50, 30), (50, 60), (20, 60): the top and
    bottom arcs bulge poleward, so between the bottom arc's highest point and
    z = sin 60 the cell spans exactly the 30 degrees between its meridians."""
    cell = [_sph(20, 30), _sph(50, 30), _sph(50, 60), _sph(20, 60)]
    ztop = math.sin(math.radians(60))
    zb = max(areas.breakpoints([_sph(20, 30), _sph(50, 30)]))  # bottom arc's apex
    assert zb > math.sin(math.radians(30))
    lat = list(np.linspace(zb + 1e-3, ztop, 6))
    A = areas.band_areas(cell, lat)
    np.testing.assert_allclose(A, math.radians(30) * np.diff(lat), rtol=1e-14, atol=0)


@pytest.mark.parametrize("m,colat", [(5, 20.0), (8, 3.0)])
def test_polar_cap_polygon(m, colat):
    """A regular m-gon around the north pole at colatitude theta: the fan of
    isosceles triangles with apex angle g = 2 pi / m gives the area
    m * 2 atan(t^2 sin g / (1 + t^2 cos g)), t = tan(theta / 2); above the
    boundary W = 2 pi."""
    cell = [_sph(360.0 * i / m + 7.0, 90.0 - colat) for i in range(m)]
    assert areas.winding(cell) == 1
    t = math.tan(math.radians(colat) / 2)
    g = TWO_PI / m
    area = m * 2 * math.atan(t * t * math.sin(g) / (1 + t * t * math.cos(g)))
    zc = math.cos(math.radians(colat))     # the vertices' height
    zb = max(areas.breakpoints(cell))      # the arcs bulge poleward up to here
    lat = [zc - 0.05, zc - 0.01, zc, zb, zb + 0.5 * (1 - zb), 1.0]
    A = areas.band_areas(cell, lat)
    assert sum(A) == pytest.approx(area, rel=1e-14)
    assert A[0] == 0.0 and A[1] == 0.0
    np.testing.assert_allclose(A[3:], TWO_PI * np.diff(lat)[3:], rtol=1e-15)
    assert areas.cell_area(cell) == pytest.approx(area, rel=1e-14)


def test_south_polar_cap_mirrors_north():
    m, colat = 6, 10.0
    north = [_sph(360.0 * i / m, 90.0 - colat) for i in range(m)]
    south = [(x, y, -z) for (x, y, z) in reversed(north)]
    assert areas.winding(south) == -1
    lat = [-1.0, -0.995, -0.99, -0.98, -0.9]
    mlat = [-z for z in reversed(lat)]
    A_s = areas.band_areas(south, lat)
    A_n = areas.band_areas(north, mlat)
    np.testing.assert_allclose(A_s, A_n[::-1], rtol=1e-14, atol=1e-17)


def test_reflection_z():
    nodes, off, fn = W.polygon_cells(8, seed=5, radius=(0.01, 0.4))
    cells = W.cells_as_lists(nodes, off, fn)
    lat = W.latlon_latitudes(37)
    for c in cells:
        mirror = [(x, y, -z) for (x, y, z) in reversed(c)]
        A = areas.band_areas(c, lat)
        Am = areas.band_areas(mirror, [-z for z in reversed(lat)])
        np.testing.assert_allclose(A, Am[::-1], rtol=1e-13, atol=1e-17 * max(A))


def test_more_nodes_change_nothing():
    nodes, off, fn = W.polygon_cells(4, seed=11, radius=(0.05, 0.3))
    cells = W.cells_as_lists(nodes, off, fn)
    lat = W.latlon_latitudes(61)
    for c in cells:
        a16 = np.array(areas.band_areas(c, lat))
        a40 = np.array(areas.band_areas(c, lat, nodes=40))
        np.testing.assert_allclose(a16, a40, rtol=1e-14, atol=1e-16 * areas.cell_area(c))


def test_crossing_directions_follow_the_slots():
    """Slot 0 of Eq. 2.2 moves upwards along x1 -> x2: the arc's point a little
    after a slot-0 crossing is higher than the crossing's latitude."""
    from oracle import exact
    rng = np.random.default_rng(3)
    checked = 0
    for _ in range(200):
        a = rng.standard_normal(3); a /= np.linalg.norm(a)
        b = rng.standard_normal(3); b /= np.linalg.norm(b)
        z0 = float(rng.uniform(min(a[2], b[2]), max(a[2], b[2])))
        r = exact.intersect(tuple(a), tuple(b), z0)
        n = np.cross(a, b)
        for slot in range(2):
            P = np.array(r.pts[slot])
            if np.isnan(P).any():
                continue
            step = np.cross(n / np.linalg.norm(n), P)  # direction of travel
            dz = (P + 1e-6 * step)[2] - z0
            assert (dz > 0) == (slot == 0)
            checked += 1
    assert checked > 150


def test_zonal_sums_of_a_constant_field():
    nodes, off, fn = W.cubed_sphere_cells(2)
    cells = W.cells_as_lists(nodes, off, fn)
    lat = W.latlon_latitudes(5)
    fa, aa = areas.zonal_sums(cells, [3.0] * len(cells), lat)
    np.testing.assert_allclose(aa, TWO_PI * np.diff(lat), atol=1e-14)
    np.testing.assert_allclose(fa, 3.0 * np.array(aa), rtol=1e-15)
