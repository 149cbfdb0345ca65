"""Seeded synthetic inputs for the arc x latitude workloads (host, numpy).

This module draws inputs only: it holds none of the intersection method's
arithmetic (no normals, no Eq. 2.2). Arcs are built from the great-circle
parametrisation x(t) = cos(t) a + sin(t) b with orthonormal a, b, which also
gives an arc's z-range for sampling latitudes inside it. Both the oracle side
(tests) and the CUDA side (tests, bench) take their inputs from here.

The paper's own datasets (MPFR-sampled latitude bands, and the near-equator
ill-conditioned set of Sec. 7) are not available; these generators stand in
for them with the same structure:

* ``uniform_arcs``    endpoints uniform on the sphere, arc length U(0, pi/2),
                      one latitude drawn uniformly in the arc's z-range
                      (10^4 arcs: the small parity workload).
* ``stress_arcs``     the ill-conditioned mix (10^6 arcs): 40 % short arcs
                      (length log-uniform 1e-10..1e-2 rad), 30 % latitudes
                      within 1e-12 of the arc's z-extremum (a third of them
                      in the paper's near-equator band of Sec. 7), 20 %
                      near-pole arcs (|z| > 1 - 1e-6), 10 % near-antipodal
                      endpoints.
* ``mixed_arcs``      90 % uniform + 10 % stress, generated in fixed chunks so
                      any sample can be regenerated alone (2x10^8 arcs).
* ``cubed_sphere_edges`` + ``latlon_latitudes`` the regridding workload.
* ``ragged_meshes``   independent random polygon meshes with per-mesh
                      latitude grids.
* ``cubed_sphere_cells`` / ``polygon_cells``  node-indexed cells (counter-
                      clockwise seen from outside) for the band-area step.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 20251009
CHUNK = 1 << 20  # arcs per independently seeded chunk (mixed_arcs)


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _random_unit(rng, n):
    return _unit(rng.standard_normal((n, 3)))


def _orthonormal_partner(rng, a):
    """A random unit vector perpendicular to each row of a."""
    g = rng.standard_normal(a.shape)
    g -= np.sum(g * a, axis=1, keepdims=True) * a
    return _unit(g)


def _arc_z_range(a, b, L):
    """z-range of the arc x(t) = cos t a + sin t b, t in [0, L] (L < pi + eps)."""
    az, bz = a[:, 2], b[:, 2]
    amp = np.hypot(az, bz)
    tmax = np.mod(np.arctan2(bz, az), 2 * np.pi)  # z(t) = amp cos(t - tmax)
    tmin = np.mod(tmax + np.pi, 2 * np.pi)
    z_end0 = az
    z_end1 = np.cos(L) * az + np.sin(L) * bz
    zhi = np.maximum(z_end0, z_end1)
    zlo = np.minimum(z_end0, z_end1)
    zhi = np.where(tmax <= L, amp, zhi)
    zlo = np.where(tmin <= L, -amp, zlo)
    return zlo, zhi


def _arcs_from_length(rng, L):
    n = L.shape[0]
    a = _random_unit(rng, n)
    b = _orthonormal_partner(rng, a)
    x1 = a
    x2 = np.cos(L)[:, None] * a + np.sin(L)[:, None] * b
    return x1, x2, a, b


def _z_in_range(rng, a, b, L):
    zlo, zhi = _arc_z_range(a, b, L)
    return zlo + rng.random(L.shape[0]) * (zhi - zlo)


def uniform_arcs(n: int, seed: int = DEFAULT_SEED):
    """(A, B, z0): endpoints uniform on S^2, length U(0, pi/2), z0 in the arc's z-range."""
    rng = np.random.default_rng(seed)
    L = rng.random(n) * (np.pi / 2)
    x1, x2, a, b = _arcs_from_length(rng, L)
    z0 = _z_in_range(rng, a, b, L)
    return x1, x2, z0


def _short(rng, n):
    L = 10.0 ** rng.uniform(-10, -2, n)
    x1, x2, a, b = _arcs_from_length(rng, L)
    return x1, x2, _z_in_range(rng, a, b, L)


def _tangent(rng, n):
    """Arcs containing their highest point; z0 just below it."""
    n_band = n // 3
    apex = _random_unit(rng, n)
    apex[:, 2] = np.abs(apex[:, 2])
    # the paper's near-equator band (0, 1e-4 deg]: apex latitude in that band
    band_z = np.sin(np.deg2rad(rng.uniform(1e-7, 1e-4, n_band)))
    lon = rng.uniform(0, 2 * np.pi, n_band)
    cz = np.sqrt(1.0 - band_z * band_z)
    apex[:n_band] = np.stack([cz * np.cos(lon), cz * np.sin(lon), band_z], axis=1)
    ez = np.array([0.0, 0.0, 1.0])
    h = _unit(np.cross(np.broadcast_to(ez, apex.shape), apex))  # horizontal tangent
    t1 = rng.uniform(1e-3, np.pi / 4, n)
    t2 = rng.uniform(1e-3, np.pi / 4, n)
    x1 = np.cos(t1)[:, None] * apex - np.sin(t1)[:, None] * h
    x2 = np.cos(t2)[:, None] * apex + np.sin(t2)[:, None] * h
    r = 10.0 ** rng.uniform(-16, -12, n)
    r[:n_band] = apex[:n_band, 2] * 10.0 ** rng.uniform(-15, -2, n_band)
    z0 = apex[:, 2] - r
    # half of them mirrored to the southern hemisphere (z -> -z)
    flip = rng.random(n) < 0.5
    flip[:n_band] = False
    for v in (x1, x2):
        v[flip, 2] = -v[flip, 2]
    z0[flip] = -z0[flip]
    return x1, x2, z0


def _near_pole(rng, n):
    def cap_points(m):
        cz = 1.0 - rng.random(m) * 1e-6
        sz = np.sqrt((1.0 - cz) * (1.0 + cz))
        lon = rng.uniform(0, 2 * np.pi, m)
        return np.stack([sz * np.cos(lon), sz * np.sin(lon), cz], axis=1)
    x1 = cap_points(n)
    x2 = cap_points(n)
    south = rng.random(n) < 0.5
    x1[south, 2] *= -1
    x2[south, 2] *= -1
    z0 = _z_for_endpoints(rng, x1, x2)
    return x1, x2, z0


def _z_for_endpoints(rng, x1, x2):
    """z0 uniform in the z-range of the minor arc x1 -> x2."""
    a = _unit(x1)
    g = x2 - np.sum(x2 * a, axis=1, keepdims=True) * a
    b = _unit(g)
    L = np.arctan2(np.linalg.norm(g, axis=1), np.sum(x2 * a, axis=1))
    return _z_in_range(rng, a, b, L)


def _antipodal(rng, n):
    x1 = _random_unit(rng, n)
    d = _random_unit(rng, n) * (10.0 ** rng.uniform(-12, -4, n))[:, None]
    x2 = _unit(-x1 + d)
    z0 = _z_for_endpoints(rng, x1, x2)
    return x1, x2, z0


STRESS_CLASSES = (("short", 0.4), ("tangent", 0.3), ("pole", 0.2), ("antipodal", 0.1))


def stress_arcs(n: int, seed: int = DEFAULT_SEED + 1, return_class: bool = False):
    """Ill-conditioned mix: 40 % short, 30 % near-tangent, 20 % near-pole, 10 % near-antipodal."""
    rng = np.random.default_rng(seed)
    counts = [int(round(n * w)) for _, w in STRESS_CLASSES]
    counts[0] += n - sum(counts)
    makers = {"short": _short, "tangent": _tangent, "pole": _near_pole, "antipodal": _antipodal}
    parts, cls = [], []
    for (name, _), m in zip(STRESS_CLASSES, counts):
        if m > 0:
            parts.append(makers[name](rng, m))
            cls.append(np.full(m, [c for c, _ in STRESS_CLASSES].index(name), dtype=np.int8))
    x1 = np.concatenate([p[0] for p in parts])
    x2 = np.concatenate([p[1] for p in parts])
    z0 = np.concatenate([p[2] for p in parts])
    klass = np.concatenate(cls)
    perm = rng.permutation(n)
    out = (np.ascontiguousarray(x1[perm]), np.ascontiguousarray(x2[perm]),
           np.ascontiguousarray(z0[perm]))
    if return_class:
        return out + (klass[perm],)
    return out


def mixed_chunk(k: int, seed: int = DEFAULT_SEED + 4, size: int = CHUNK):
    """Chunk k of the 90/10 uniform/stress mix (regenerable on its own)."""
    ss = np.random.SeedSequence([seed, k])
    s_uni, s_str, s_mix = ss.generate_state(3)
    n_str = size // 10
    u = uniform_arcs(size - n_str, seed=int(s_uni))
    s = stress_arcs(n_str, seed=int(s_str))
    perm = np.random.default_rng(int(s_mix)).permutation(size)
    return tuple(np.ascontiguousarray(np.concatenate([a, b])[perm]) for a, b in zip(u, s))


def mixed_arcs(n: int, seed: int = DEFAULT_SEED + 4):
    """n arcs of the 90/10 mix, as consecutive chunks of CHUNK arcs."""
    A = np.empty((n, 3))
    B = np.empty((n, 3))
    z = np.empty(n)
    for k in range((n + CHUNK - 1) // CHUNK):
        lo, hi = k * CHUNK, min(n, (k + 1) * CHUNK)
        a, b, c = mixed_chunk(k, seed)
        A[lo:hi], B[lo:hi], z[lo:hi] = a[:hi - lo], b[:hi - lo], c[:hi - lo]
    return A, B, z


# ------------------------------------------------------------------ meshes --
def cubed_sphere_edges(N: int):
    """Edges of an equiangular gnomonic cubed sphere with N x N cells per face.

    Each face contributes N(N+1) edges along each grid direction, so the mesh
    has 12 N (N+1) edges (face-boundary edges appear once per adjacent face).
    Returns (A, B) as (E, 3) arrays of unit vectors.
    """
    ang = -np.pi / 4 + (np.pi / 2) * np.arange(N + 1) / N
    t = np.tan(ang)
    u, v = np.meshgrid(t, t, indexing="ij")  # (N+1, N+1)
    one = np.ones_like(u)
    faces = [(one, u, v), (-one, -u, v), (-u, one, v), (u, -one, v), (-v, u, one), (v, u, -one)]
    A_parts, B_parts = [], []
    for fx, fy, fz in faces:
        P = _unit(np.stack([fx, fy, fz], axis=-1))  # (N+1, N+1, 3)
        A_parts += [P[:-1, :, :].reshape(-1, 3), P[:, :-1, :].reshape(-1, 3)]
        B_parts += [P[1:, :, :].reshape(-1, 3), P[:, 1:, :].reshape(-1, 3)]
    return (np.ascontiguousarray(np.concatenate(A_parts)),
            np.ascontiguousarray(np.concatenate(B_parts)))


def latlon_latitudes(n_lat: int):
    """z of n_lat equally spaced latitudes from -90 to +90 degrees (ascending)."""
    deg = -90.0 + 180.0 * np.arange(n_lat) / (n_lat - 1)
    z = np.sin(np.deg2rad(deg))
    z[0], z[-1] = -1.0, 1.0
    return z


def _fibonacci_points(m):
    i = np.arange(m) + 0.5
    z = 1.0 - 2.0 * i / m
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * np.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def polygon_mesh(rng, n_edges: int):
    """Independent small polygons (3-12 vertices) around jittered Fibonacci points.

    Returns (A, B) edge endpoint arrays with exactly n_edges rows.
    """
    kmean = 7.5
    m = max(1, int(math.ceil(n_edges / kmean)))
    centres = _fibonacci_points(m)
    spacing = math.sqrt(4 * math.pi / m)
    centres = _unit(centres + 0.3 * spacing * rng.standard_normal((m, 3)))
    k = rng.integers(3, 13, m)
    tot = int(k.sum())
    while tot < n_edges:  # top up with more polygons if the draw fell short
        extra = rng.integers(3, 13, 8)
        k = np.concatenate([k, extra])
        centres = np.concatenate([centres, _random_unit(rng, 8)])
        tot = int(k.sum())
    # tangent frame at each centre
    e1 = _orthonormal_partner(rng, centres)
    e2 = np.cross(centres, e1)
    poly = np.repeat(np.arange(k.size), k)
    first = np.concatenate([[0], np.cumsum(k)[:-1]])
    j = np.arange(tot) - first[poly]
    ang = 2 * np.pi * (j + 0.3 * rng.random(tot)) / k[poly]
    rad = 0.5 * spacing
    V = _unit(centres[poly] + rad * (np.cos(ang)[:, None] * e1[poly] + np.sin(ang)[:, None] * e2[poly]))
    nxt = np.where(j + 1 == k[poly], first[poly], np.arange(tot) + 1)
    A = V[:n_edges]
    B = V[nxt][:n_edges]
    return np.ascontiguousarray(A), np.ascontiguousarray(B)


def ragged_sizes(n_mesh: int, e_min: float, e_max: float, seed: int = DEFAULT_SEED + 3,
                 lat_min: int = 180, lat_max: int = 2881):
    """Edge counts (log-uniform in [e_min, e_max]) and latitude counts (uniform
    in [lat_min, lat_max]) of a mesh batch."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0]))
    E = np.exp(rng.uniform(math.log(e_min), math.log(e_max), n_mesh)).astype(np.int64)
    E = np.maximum(E, 1)
    L = rng.integers(lat_min, lat_max + 1, n_mesh)
    return E, L


def ragged_mesh(args):
    """Mesh m of a batch, (m, n_edges, seed) -> (A, B): seeded on its own, so
    the meshes of a batch can be generated independently (in parallel)."""
    m, n_edges, seed = args
    rng = np.random.default_rng(np.random.SeedSequence([seed, 1, int(m)]))
    return polygon_mesh(rng, int(n_edges))


def ragged_meshes(n_mesh: int, e_min: float, e_max: float, seed: int = DEFAULT_SEED + 3,
                  lat_min: int = 180, lat_max: int = 2881):
    """A batch of independent polygon meshes with per-mesh latitude grids.

    Edge counts are log-uniform in [e_min, e_max]; latitude counts uniform in
    [lat_min, lat_max]. Returns dict with A, B (E,3), edge_offsets (M+1,),
    lat_z (sum L,), lat_offsets (M+1,).
    """
    E, L = ragged_sizes(n_mesh, e_min, e_max, seed, lat_min, lat_max)
    A_parts, B_parts, Z_parts = [], [], []
    for m in range(n_mesh):
        a, b = ragged_mesh((m, E[m], seed))
        A_parts.append(a)
        B_parts.append(b)
        Z_parts.append(latlon_latitudes(int(L[m])))
    edge_offsets = np.concatenate([[0], np.cumsum(E)]).astype(np.int64)
    lat_offsets = np.concatenate([[0], np.cumsum(L)]).astype(np.int64)
    return {"A": np.ascontiguousarray(np.concatenate(A_parts)),
            "B": np.ascontiguousarray(np.concatenate(B_parts)),
            "edge_offsets": edge_offsets,
            "lat_z": np.ascontiguousarray(np.concatenate(Z_parts)),
            "lat_offsets": lat_offsets}


# ---------------------------------------------------------- arc x arc pairs --
def _arc_through(p, d, length, frac):
    """Endpoints of the arc x(t) = cos t p + sin t d, t in [-frac L, (1 - frac) L]."""
    t0 = (-frac * length)[:, None]
    t1 = ((1.0 - frac) * length)[:, None]
    return np.cos(t0) * p + np.sin(t0) * d, np.cos(t1) * p + np.sin(t1) * d


ARC_CLASSES = (("uniform", 0.5), ("short", 0.15), ("parallel", 0.15), ("endpoint", 0.1),
               ("miss", 0.1))


def arc_pairs(n: int, seed: int = DEFAULT_SEED + 5, return_class: bool = False):
    """Pairs of great circle arcs (a1, a2), (b1, b2) built around a crossing
    point p: both circles pass through p, at an angle; each arc covers p at a
    fraction of its length, except for the 'miss' class, whose arc b stops
    short of p. Classes: 50 % uniform (lengths U(0, pi/2), angle U(0, pi)),
    15 % short arcs (length log-uniform 1e-10..1e-2 rad), 15 % nearly parallel
    circles (angle log-uniform 1e-12..1e-3), 10 % crossings near an endpoint
    (fraction log-uniform 1e-12..1e-3 from either end), 10 % misses."""
    rng = np.random.default_rng(seed)
    counts = [int(round(n * w)) for _, w in ARC_CLASSES]
    counts[0] += n - sum(counts)
    klass = np.concatenate([np.full(c, i, dtype=np.int8) for i, c in enumerate(counts)])
    klass = klass[rng.permutation(n)]
    p = _random_unit(rng, n)
    d1 = _orthonormal_partner(rng, p)
    d1x = np.cross(p, d1)
    ang = rng.uniform(0.0, np.pi, n)
    par = klass == 2
    ang[par] = 10.0 ** rng.uniform(-12, -3, par.sum()) * np.where(rng.random(par.sum()) < 0.5, 1, -1)
    d2 = np.cos(ang)[:, None] * d1 + np.sin(ang)[:, None] * d1x
    La = rng.uniform(0.0, np.pi / 2, n)
    Lb = rng.uniform(0.0, np.pi / 2, n)
    sh = klass == 1
    La[sh] = 10.0 ** rng.uniform(-10, -2, sh.sum())
    Lb[sh] = 10.0 ** rng.uniform(-10, -2, sh.sum())
    fa = rng.random(n)
    fb = rng.random(n)
    ep = klass == 3
    tiny = 10.0 ** rng.uniform(-12, -3, ep.sum())
    fb[ep] = np.where(rng.random(ep.sum()) < 0.5, tiny, 1.0 - tiny)
    ms = klass == 4
    fb[ms] = -rng.uniform(0.05, 1.0, ms.sum())  # arc b ends before reaching p
    a1, a2 = _arc_through(p, d1, La, fa)
    b1, b2 = _arc_through(p, d2, Lb, fb)
    out = tuple(np.ascontiguousarray(v) for v in (a1, a2, b1, b2))
    if return_class:
        return out + (klass,)
    return out


# ---- node-indexed cells for the band-area (zonal-mean) step -------------------
def _tan_grid(N: int):
    """tan of N + 1 equiangular angles from -pi/4 to pi/4, odd-symmetric, with
    exact ends: T[0] = -1, T[N] = 1, T[N - i] = -T[i]."""
    t = np.tan(-np.pi / 4 + (np.pi / 2) * np.arange(N + 1) / N)
    half = (N + 1) // 2
    t[N + 1 - half:] = -t[:half][::-1]
    if N % 2 == 0:
        t[N // 2] = 0.0
    t[0], t[N] = -1.0, 1.0
    return t


def cubed_sphere_cells(N: int):
    """Equiangular gnomonic cubed sphere as node-indexed quadrilaterals.

    Every node is a point (T[i], T[j], T[k]) of the cube surface's lattice
    (i, j, k in 0..N, one of them 0 or N), normalised; a node shared by
    several faces of the cube is stored once, so neighbouring cells share
    their edges bit for bit. Cells run counter-clockwise seen from outside.
    For even N the poles are nodes; for odd N each pole lies inside a cell.

    Returns (nodes (6 N^2 + 2, 3) float64, face_offsets (6 N^2 + 1,) int64,
    face_nodes (24 N^2,) int32).
    """
    T = _tan_grid(N)
    n1 = N + 1
    a, b = np.meshgrid(np.arange(n1), np.arange(n1), indexing="ij")
    full = np.full_like(a, N)
    zero = np.zeros_like(a)
    # (i, j, k) lattice indices per cube face, with in-face axes u, v such that
    # u x v is the outward normal (so increasing (u, v) order is counter-clockwise)
    faces = [(full, a, b),   # +x: u = y, v = z
             (zero, b, a),   # -x: u = z, v = y
             (b, full, a),   # +y: u = z, v = x
             (a, zero, b),   # -y: u = x, v = z
             (a, b, full),   # +z: u = x, v = y
             (b, a, zero)]   # -z: u = y, v = x
    keys = np.concatenate([((i * n1 + j) * n1 + k).ravel() for i, j, k in faces])
    uniq, inv = np.unique(keys, return_inverse=True)
    ii, rem = np.divmod(uniq, n1 * n1)
    jj, kk = np.divmod(rem, n1)
    P = np.stack([T[ii], T[jj], T[kk]], axis=1)
    nodes = np.ascontiguousarray(P / np.sqrt(np.sum(P * P, axis=1, keepdims=True)))
    inv = inv.reshape(6, n1, n1).astype(np.int32)
    quads = np.stack([inv[:, :-1, :-1], inv[:, 1:, :-1], inv[:, 1:, 1:], inv[:, :-1, 1:]],
                     axis=-1)
    face_nodes = np.ascontiguousarray(quads.reshape(-1))
    face_offsets = 4 * np.arange(6 * N * N + 1, dtype=np.int64)
    return nodes, face_offsets, face_nodes


def polygon_cells(n_cells: int, seed: int = DEFAULT_SEED + 6, radius=(1e-3, 0.3),
                  kmin: int = 3, kmax: int = 12, star: float = 0.3):
    """Independent random star-shaped polygons (kmin..kmax vertices), centres
    uniform on the sphere, radius log-uniform in [radius], vertex radii
    jittered by +-star (non-convex for star > 0), counter-clockwise.

    Returns (nodes, face_offsets, face_nodes) like ``cubed_sphere_cells``
    (each cell owns its nodes).
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 7]))
    c = _random_unit(rng, n_cells)
    e1 = _orthonormal_partner(rng, c)
    e2 = np.cross(c, e1)  # e1 x e2 = c: increasing angle is counter-clockwise
    k = rng.integers(kmin, kmax + 1, n_cells)
    rad = np.exp(rng.uniform(math.log(radius[0]), math.log(radius[1]), n_cells))
    tot = int(k.sum())
    cell = np.repeat(np.arange(n_cells), k)
    first = np.concatenate([[0], np.cumsum(k)[:-1]])
    j = np.arange(tot) - first[cell]
    ang = 2 * np.pi * (j + 0.4 * rng.random(tot)) / k[cell]
    r = rad[cell] * (1.0 + star * rng.uniform(-1.0, 1.0, tot))
    V = c[cell] + np.tan(r)[:, None] * (np.cos(ang)[:, None] * e1[cell] +
                                        np.sin(ang)[:, None] * e2[cell])
    nodes = np.ascontiguousarray(_unit(V))
    face_offsets = np.concatenate([[0], np.cumsum(k)]).astype(np.int64)
    return nodes, face_offsets, np.arange(tot, dtype=np.int32)


def cells_as_lists(nodes, face_offsets, face_nodes, which=None):
    """Cells as lists of vertex tuples (for the oracle), optionally a subset."""
    idx = range(len(face_offsets) - 1) if which is None else which
    out = []
    for f in idx:
        ids = face_nodes[face_offsets[f]:face_offsets[f + 1]]
        out.append([tuple(float(x) for x in nodes[i]) for i in ids])
    return out


# ------------------------------------------------- near-boundary arcs ---------
# Pythagorean triples (p, q, r): a rotation about the z-axis by atan2(q, p),
# scaled by r, maps integer vectors to integer vectors exactly (directions, and
# so latitudes, are all that the intersection depends on).
_PYTHAGOREAN = ((3, 4, 5), (5, 12, 13), (8, 15, 17), (7, 24, 25), (20, 21, 29),
                (12, 35, 37), (9, 40, 41), (28, 45, 53), (11, 60, 61), (33, 56, 65))

NEAR_CLASSES = (("tangent", 0.3), ("tangent_rotated", 0.2), ("endpoint_offset", 0.4),
                ("endpoint_z", 0.1))


def _convergents(x, max_den: int):
    """Continued-fraction convergents p/q of the positive Fraction x with q <= max_den."""
    from fractions import Fraction
    out = []
    p0, q0, p1, q1 = 0, 1, 1, 0
    num, den = x.numerator, x.denominator
    while den:
        a, r = divmod(num, den)
        p0, p1 = p1, a * p1 + p0
        q0, q1 = q1, a * q1 + q0
        if q1 > max_den:
            break
        out.append(Fraction(p1, q1))
        num, den = den, r
    return out


def _near_tangent_one(rng, rotated: bool, log2_range=(80.0, 110.0)):
    """One arc whose great circle is tangent to the latitude z0 to within
    |s^2| / |n_xy|^2 = 2^-e, e in log2_range (where constructible).

    The arc lies in the plane through the z-axis direction (a, 0, b) and the
    y-axis: x1 = (a, Y1, b), x2 = (a, -Y2, b), whose highest point has height
    b / sqrt(a^2 + b^2). With z0 fixed, a / b is taken from the convergents of
    sqrt(1 - z0^2) / z0, so that height approaches z0 as closely as integers
    a, b < 2^52 allow; the relative gap of the squared heights is then an
    exact rational, and a convergent whose gap lands in the range is kept.
    The rotated variant keeps a, b, Y < 2^46 and turns the plane about the
    z-axis by a Pythagorean angle, exactly in integers.
    """
    from fractions import Fraction
    lim = 1 << (45 if rotated else 52)
    while True:
        z0 = float(rng.uniform(0.02, 0.98))
        zf = Fraction(z0)
        t2 = (1 - zf * zf) / (zf * zf)             # (a / b)^2 at exact tangency
        k = 320
        t = Fraction(math.isqrt((t2.numerator << (2 * k)) // t2.denominator), 1 << k)
        picks = []
        for c in _convergents(t, lim):
            a, b = c.numerator, c.denominator
            if a >= lim or a == 0:
                continue
            gap = (1 - zf * zf) - zf * zf * Fraction(a * a, b * b)   # s^2 / |n_xy|^2
            if gap == 0:
                continue
            e = -math.log2(abs(gap.numerator) / gap.denominator)
            if log2_range[0] <= e <= log2_range[1]:
                picks.append((a, b))
        if picks:
            a, b = picks[int(rng.integers(len(picks)))]
            break
    if rotated:
        y1 = int(b * rng.uniform(0.05, 1.5)) + 1
        y2 = int(b * rng.uniform(0.05, 1.5)) + 1
        p, q, r = _PYTHAGOREAN[int(rng.integers(len(_PYTHAGOREAN)))]
        v1 = [p * a - q * y1, q * a + p * y1, r * b]
        v2 = [p * a + q * y2, q * a - p * y2, r * b]
    else:
        y1 = float(b) * rng.uniform(0.05, 1.5)
        y2 = float(b) * rng.uniform(0.05, 1.5)
        v1 = [a, y1, b]
        v2 = [a, -y2, b]
    x1 = np.array(v1, dtype=np.float64)
    x2 = np.array(v2, dtype=np.float64)
    # exact symmetries of the square about the z-axis
    if rng.random() < 0.5:
        x1[[0, 1]] = x1[[1, 0]]
        x2[[0, 1]] = x2[[1, 0]]
    for ax in (0, 1):
        if rng.random() < 0.5:
            x1[ax], x2[ax] = -x1[ax], -x2[ax]
    if rng.random() < 0.5:                          # mirror to the south
        x1[2], x2[2], z0 = -x1[2], -x2[2], -z0
    # powers of two bring the endpoints near unit length (exact)
    x1 = np.ldexp(x1, -int(np.frexp(np.abs(x1).max())[1]))
    x2 = np.ldexp(x2, -int(np.frexp(np.abs(x2).max())[1]))
    if rng.random() < 0.5:
        x1, x2 = x2, x1
    return x1, x2, z0


def near_boundary_arcs(n: int, seed: int = DEFAULT_SEED + 7, return_class: bool = False):
    """Arcs at the two decision boundaries of the method (Sec. 2: whether the
    circles meet, and whether a candidate lies between the endpoints):

    * ``tangent`` (30 %): great circles tangent to their latitude to within
      |s^2| / |n_xy|^2 of 2^-80 .. 2^-104 (integer-ratio construction, see
      _near_tangent_one), both signs, with the apex inside the arc;
    * ``tangent_rotated`` (20 %): the same, turned about the z-axis by a
      Pythagorean angle (gaps 2^-80 .. about 2^-92);
    * ``endpoint_offset`` (40 %): arcs of length U(0.01, pi/2) whose latitude
      passes 2^-45 .. 2^-30 rad (log-uniform) inside or outside one endpoint
      along the arc (placed where the height changes by >= 0.1 per radian);
    * ``endpoint_z`` (10 %): z0 equal to one endpoint's z, bit for bit
      (the candidate sits within rounding of the endpoint), a fifth of them
      with an exactly unit endpoint on the equator and z0 = 0 (the candidate
      is that endpoint).
    """
    rng = np.random.default_rng(seed)
    counts = [int(round(n * w)) for _, w in NEAR_CLASSES]
    counts[0] += n - sum(counts)
    klass = np.concatenate([np.full(c, i, dtype=np.int8) for i, c in enumerate(counts)])
    klass = klass[rng.permutation(n)]
    A = np.empty((n, 3))
    B = np.empty((n, 3))
    z = np.empty(n)
    for i in range(n):
        k = NEAR_CLASSES[klass[i]][0]
        if k in ("tangent", "tangent_rotated"):
            A[i], B[i], z[i] = _near_tangent_one(rng, k == "tangent_rotated")
            continue
        while True:
            a = _random_unit(rng, 1)
            b = _orthonormal_partner(rng, a)
            a, b = a[0], b[0]
            L = float(rng.uniform(0.01, np.pi / 2))
            end = int(rng.integers(2))
            te = 0.0 if end == 0 else L
            slope = -math.sin(te) * a[2] + math.cos(te) * b[2]
            if abs(slope) >= 0.1:
                break
        x1 = a
        x2 = math.cos(L) * a + math.sin(L) * b
        if k == "endpoint_offset":
            d = 2.0 ** rng.uniform(-45, -30) * (1 if rng.random() < 0.5 else -1)
            t = d if end == 0 else L - d                 # d > 0: inside the arc
            if end == 0:
                zz = a[2] + d * b[2] - 0.5 * d * d * a[2]
            else:
                zz = math.cos(t) * a[2] + math.sin(t) * b[2]
        else:
            if rng.random() < 0.2:
                ax = int(rng.integers(2))
                x1 = np.zeros(3)
                x1[ax] = 1.0 if rng.random() < 0.5 else -1.0
                zz = 0.0
            else:
                zz = (x1 if end == 0 else x2)[2]
        A[i], B[i], z[i] = x1, x2, zz
    out = (np.ascontiguousarray(A), np.ascontiguousarray(B), np.ascontiguousarray(z))
    if return_class:
        return out + (klass,)
    return out
