"""Seeded synthetic inputs: triangulated city scenes and ray batches.

This module only draws inputs.  It holds none of the method's arithmetic (no
bounding boxes, no split cost, no intersection test), so both the CUDA path and
the CPU checker can be fed from it without sharing any of the method.

The paper's scenes (an indoor study room and a university campus, Sec. IV.A)
were authored in SketchUp and are not available; the generators below produce
scenes of the same kind: buildings stored as triangular facets (Sec. II.A)
standing on a flat ground, with transmitters a few tens of metres above it.

Rays are launched as in Sec. III.A: from a source point towards the vertices
of a subdivided regular icosahedron (12 vertices, 20 faces, each face split
into f*f smaller triangles), or, where a workload asks for it, towards the
points of a Fibonacci sphere.  Directions are formed in float64 and rounded
once to float32.

Array conventions (all C-contiguous):
  tris  float32 [T, 3, 3]   vertex k of triangle i is tris[i, k, :]
  rays  float32 [R, 8]      (ox, oy, oz, tmin, dx, dy, dz, tmax)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# scene containers
# --------------------------------------------------------------------------


@dataclass
class Scene:
    """A triangle soup plus the facts a workload needs about it."""

    tris: np.ndarray               # float32 [T, 3, 3]
    area: tuple                    # (xmin, ymin, xmax, ymax) of the ground
    n_buildings: int
    seed: int
    name: str = ""
    tx: list = field(default_factory=list)   # transmitter positions (float64 [3])

    @property
    def n_tri(self) -> int:
        return int(self.tris.shape[0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _ground(xmin, ymin, xmax, ymax):
    """Two triangles covering the rectangle at z = 0 (normal +z)."""
    a = (xmin, ymin, 0.0)
    b = (xmax, ymin, 0.0)
    c = (xmax, ymax, 0.0)
    d = (xmin, ymax, 0.0)
    return [(a, b, c), (a, c, d)]


def _box(x0, y0, x1, y1, h):
    """12 triangles of an axis-aligned box [x0,x1]x[y0,y1]x[0,h], outward winding."""
    p = [(x0, y0, 0.0), (x1, y0, 0.0), (x1, y1, 0.0), (x0, y1, 0.0),
         (x0, y0, h), (x1, y0, h), (x1, y1, h), (x0, y1, h)]
    quads = [(0, 3, 2, 1),   # bottom, normal -z
             (4, 5, 6, 7),   # top, +z
             (0, 1, 5, 4),   # y = y0, -y
             (1, 2, 6, 5),   # x = x1, +x
             (2, 3, 7, 6),   # y = y1, +y
             (3, 0, 4, 7)]   # x = x0, -x
    out = []
    for q in quads:
        out.append((p[q[0]], p[q[1]], p[q[2]]))
        out.append((p[q[0]], p[q[2]], p[q[3]]))
    return out


def _prism(poly_xy, h):
    """Closed prism over a convex CCW polygon: 2n wall + 2(n-2) cap triangles."""
    n = len(poly_xy)
    bot = [(float(x), float(y), 0.0) for x, y in poly_xy]
    top = [(float(x), float(y), float(h)) for x, y in poly_xy]
    out = []
    for i in range(n):
        j = (i + 1) % n
        out.append((bot[i], bot[j], top[j]))
        out.append((bot[i], top[j], top[i]))
    for i in range(1, n - 1):          # roof fan, normal +z
        out.append((top[0], top[i], top[i + 1]))
    for i in range(1, n - 1):          # floor fan, normal -z
        out.append((bot[0], bot[i + 1], bot[i]))
    return out


# --------------------------------------------------------------------------
# cities
# --------------------------------------------------------------------------


def tiny_city(seed: int = 1, n_buildings: int = 64, size: float = 200.0,
              tx=(100.0, 100.0, 30.0)) -> Scene:
    """Axis-aligned box buildings on a square ground (64 boxes -> 770 triangles).

    Footprints are squares with side U(8, 25) m placed uniformly inside the
    area, heights U(10, 40) m.  A footprint that would contain the
    transmitter's (x, y) is redrawn, so the transmitter is never inside a
    building.
    """
    rng = _rng(seed)
    tris = []
    placed = 0
    while placed < n_buildings:
        side = rng.uniform(8.0, 25.0)
        cx = rng.uniform(side / 2, size - side / 2)
        cy = rng.uniform(side / 2, size - side / 2)
        h = rng.uniform(10.0, 40.0)
        x0, x1 = cx - side / 2, cx + side / 2
        y0, y1 = cy - side / 2, cy + side / 2
        if x0 <= tx[0] <= x1 and y0 <= tx[1] <= y1:
            continue
        tris += _box(x0, y0, x1, y1, h)
        placed += 1
    tris += _ground(0.0, 0.0, size, size)
    arr = np.asarray(tris, dtype=np.float64).astype(np.float32)
    return Scene(arr, (0.0, 0.0, size, size), n_buildings, seed, "tiny_city",
                 [np.array(tx, dtype=np.float64)])


def _convex_footprint(rng, ngon, rmin, rmax):
    n = int(rng.integers(ngon[0], ngon[1] + 1))
    ang = np.sort(rng.uniform(0.0, 2 * math.pi, size=n))
    r = rng.uniform(rmin, rmax)
    rot = rng.uniform(0.0, math.pi)
    xy = np.stack([r * np.cos(ang + rot), r * np.sin(ang + rot)], axis=1)
    return xy, r


def prism_city(n_buildings: int, size: float, seed: int, ngon=(4, 8),
               rmin: float = 4.0, rmax: float = 12.5, clusters: int = 0,
               sigma: float = 800.0, tx_keepout=(), name: str = "prism_city") -> Scene:
    """Buildings extruded from random convex n-gon footprints on a square ground.

    n ~ U{ngon}, vertex angles sorted U(0, 2 pi) on a circle of radius
    U(rmin, rmax) m, footprint rotated U(0, pi), heights lognormal(3, 0.5) m.
    Centres are uniform over the area, or (clusters > 0) drawn from an equal
    mixture of `clusters` Gaussians with uniform centres and std `sigma`,
    clipped to the area.  Buildings may overlap.  A footprint whose circle
    covers the (x, y) of a point in `tx_keepout` is redrawn.
    """
    rng = _rng(seed)
    if clusters > 0:
        cc = rng.uniform(rmax, size - rmax, size=(clusters, 2))
    tris = []
    placed = 0
    while placed < n_buildings:
        xy, r = _convex_footprint(rng, ngon, rmin, rmax)
        if clusters > 0:
            k = int(rng.integers(0, clusters))
            c = cc[k] + rng.normal(0.0, sigma, size=2)
            c = np.clip(c, r, size - r)
        else:
            c = rng.uniform(r, size - r, size=2)
        h = float(rng.lognormal(3.0, 0.5))
        if any(math.hypot(c[0] - t[0], c[1] - t[1]) <= r for t in tx_keepout):
            continue
        tris += _prism(xy + c, h)
        placed += 1
    tris += _ground(0.0, 0.0, size, size)
    arr = np.asarray(tris, dtype=np.float64).astype(np.float32)
    return Scene(arr, (0.0, 0.0, size, size), n_buildings, seed, name,
                 [np.asarray(t, dtype=np.float64) for t in tx_keepout])


def metro_city(seed: int = 5, n_buildings: int = 300_000, size: float = 20_000.0, ngon=(8, 16),
               rmin: float = 4.0, rmax: float = 12.5, clusters: int = 20, sigma: float = 800.0) -> Scene:
    """The large metro: convex 8-16-gon prisms on a 20 x 20 km ground, centres
    from an equal mixture of 20 Gaussians (uniform centres, std 800 m, clipped),
    heights lognormal(3, 0.5) m.  Same footprint and height recipe as
    prism_city, drawn in bulk (whole arrays per quantity) so that millions of
    triangles take seconds; per prism the same triangles as _prism."""
    rng = _rng(seed)
    nb = int(n_buildings)
    cc = rng.uniform(rmax, size - rmax, size=(clusters, 2))
    ng = rng.integers(ngon[0], ngon[1] + 1, size=nb)
    ang = rng.uniform(0.0, 2 * math.pi, size=(nb, ngon[1]))
    r = rng.uniform(rmin, rmax, size=nb)
    rot = rng.uniform(0.0, math.pi, size=nb)
    k = rng.integers(0, clusters, size=nb)
    c = np.clip(cc[k] + rng.normal(0.0, sigma, size=(nb, 2)), r[:, None], size - r[:, None])
    h = rng.lognormal(3.0, 0.5, size=nb)
    # the first ng angles of each row, sorted
    ang = np.where(np.arange(ngon[1])[None, :] < ng[:, None], ang, np.inf)
    ang = np.sort(ang, axis=1)
    parts = []
    for n in range(ngon[0], ngon[1] + 1):
        sel = np.nonzero(ng == n)[0]
        if len(sel) == 0:
            continue
        a = ang[sel, :n] + rot[sel, None]
        x = c[sel, 0, None] + r[sel, None] * np.cos(a)
        y = c[sel, 1, None] + r[sel, None] * np.sin(a)
        z0 = np.zeros_like(x)
        z1 = np.broadcast_to(h[sel, None], x.shape)
        bot = np.stack([x, y, z0], axis=-1)          # [m, n, 3]
        top = np.stack([x, y, z1], axis=-1)
        i = np.arange(n)
        j = (i + 1) % n
        walls_a = np.stack([bot[:, i], bot[:, j], top[:, j]], axis=2)   # [m, n, 3, 3]
        walls_b = np.stack([bot[:, i], top[:, j], top[:, i]], axis=2)
        walls = np.stack([walls_a, walls_b], axis=2).reshape(len(sel), 2 * n, 3, 3)
        f = np.arange(1, n - 1)
        roof = np.stack([np.broadcast_to(top[:, :1], (len(sel), n - 2, 3)), top[:, f], top[:, f + 1]], axis=2)
        floor = np.stack([np.broadcast_to(bot[:, :1], (len(sel), n - 2, 3)), bot[:, f + 1], bot[:, f]], axis=2)
        parts.append((sel, np.concatenate([walls, roof, floor], axis=1).astype(np.float32)))
    # buildings in draw order
    order = np.argsort(np.concatenate([p[0] for p in parts]), kind="stable")
    per = [t for p in parts for t in p[1]]
    tris = np.concatenate([per[o] for o in order] + [np.asarray(_ground(0.0, 0.0, size, size), np.float32)])
    return Scene(tris, (0.0, 0.0, size, size), nb, seed, "metro_city", [])


def medium_city(seed: int = 2, n_buildings: int = 1000, size: float = 1000.0) -> Scene:
    """1000 convex 4-8-gon prisms on 1 x 1 km (~20k triangles), Tx at the centre, 30 m."""
    tx = (size / 2, size / 2, 30.0)
    return prism_city(n_buildings, size, seed, tx_keepout=(tx,), name="medium_city")


# --------------------------------------------------------------------------
# launch directions (Sec. III.A)
# --------------------------------------------------------------------------


def fibonacci_directions(n: int) -> np.ndarray:
    """n unit directions on a Fibonacci sphere, float64 [n, 3].

    z_i = 1 - (2i + 1)/n, azimuth_i = i * pi * (3 - sqrt 5).
    """
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * (math.pi * (3.0 - math.sqrt(5.0)))
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def icosahedron():
    """The 12 vertices (0, +-1, +-phi) and cyclic shifts, and the 20 faces.

    Faces are found as the vertex triples that are pairwise at the edge length
    (2), listed in lexicographic order of their sorted indices.
    """
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-g, g):
            v.append((0.0, a, b))
            v.append((a, b, 0.0))
            v.append((b, 0.0, a))
    v = np.asarray(v, dtype=np.float64)
    n = len(v)
    adj = np.zeros((n, n), dtype=bool)
    for i in range(n):
        for j in range(n):
            if i != j and abs(np.linalg.norm(v[i] - v[j]) - 2.0) < 1e-9:
                adj[i, j] = True
    faces = []
    for i in range(n):
        for j in range(i + 1, n):
            for k in range(j + 1, n):
                if adj[i, j] and adj[j, k] and adj[i, k]:
                    faces.append((i, j, k))
    return v, np.asarray(faces, dtype=np.int64)


def icosphere_directions(level: int) -> np.ndarray:
    """Unit directions to the vertices of an icosahedron subdivided 2**level times per edge.

    Each face is cut into f*f triangles (f = 2**level) by a planar barycentric
    grid; the grid points are shared between faces through canonical edge
    orientation, then projected to the unit sphere.  Count = 10 f^2 + 2.
    Order: the 12 corners, then the points inside each of the 30 edges, then
    the points inside each of the 20 faces.
    """
    f = 1 << level
    v, faces = icosahedron()
    pts = [v]
    edges = sorted({tuple(sorted((int(a), int(b)))) for fc in faces
                    for a, b in ((fc[0], fc[1]), (fc[1], fc[2]), (fc[0], fc[2]))})
    if f > 1:
        s = (np.arange(1, f, dtype=np.float64) / f)[:, None]
        for a, b in edges:
            pts.append(v[a] * (1.0 - s) + v[b] * s)
        for a, b, c in faces:
            ii, jj = [], []
            for i in range(1, f):
                for j in range(1, f - i):
                    ii.append(i)
                    jj.append(j)
            if ii:
                wi = np.asarray(ii, dtype=np.float64)[:, None] / f
                wj = np.asarray(jj, dtype=np.float64)[:, None] / f
                pts.append(v[a] * (1.0 - wi - wj) + v[b] * wi + v[c] * wj)
    p = np.concatenate(pts, axis=0)
    return p / np.linalg.norm(p, axis=1, keepdims=True)


def icosphere_launch_order(level: int) -> np.ndarray:
    """Index (in icosphere_directions' order) of the direction in each slot of
    an icosphere launch in tile order, int64 [10 f^2 + 2].

    Corners and edge points keep their order.  Each face's interior (rows
    i = 1 .. f-2 of f-1-i points j = 1 .. f-1-i) is cut into bands of 8 rows;
    a band lists the columns all 8 of its rows hold as tiles of 8 rows x 4
    columns (tile after tile, row by row inside a tile) and the rest of its
    rows row by row; even bands (counted from 0) run tiles then rest, odd
    bands rest then the tiles from the last to the first; the rows after the
    last full band follow row by row.
    """
    f = 1 << level
    n = 10 * f * f + 2
    head = 12 + 30 * (f - 1)
    per_face = (f - 1) * (f - 2) // 2
    def row_start(i):                      # first point of row i in a face
        return (i - 1) * (f - 1) - (i - 1) * i // 2
    local = []
    nb = (f - 2) // 8 if f >= 2 else 0
    for r in range(nb):
        rows = [8 * r + 1 + k for k in range(8)]
        lens = [f - 1 - i for i in rows]
        nblk = lens[-1] // 4
        tiles = [[row_start(rows[k]) + 4 * b + c for k in range(8) for c in range(4)] for b in range(nblk)]
        rest = [row_start(rows[k]) + j - 1 for k in range(8) for j in range(4 * nblk + 1, lens[k] + 1)]
        if r % 2 == 0:
            local += [x for t in tiles for x in t] + rest
        else:
            local += rest + [x for t in reversed(tiles) for x in t]
    for i in range(8 * nb + 1, f - 1):
        local += [row_start(i) + j - 1 for j in range(1, f - i)]
    local = np.asarray(local, dtype=np.int64)
    assert local.size == max(per_face, 0)
    perm = np.arange(n, dtype=np.int64)
    for fc in range(20):
        perm[head + fc * per_face:head + (fc + 1) * per_face] = head + fc * per_face + local
    return perm


def make_rays(origin, dirs, tmin: float = 0.0, tmax: float = np.inf) -> np.ndarray:
    """Pack rays from one origin as float32 [R, 8] = (o, tmin, d, tmax)."""
    dirs = np.asarray(dirs, dtype=np.float64)
    r = np.empty((dirs.shape[0], 8), dtype=np.float32)
    r[:, 0:3] = np.asarray(origin, dtype=np.float64)[None, :].astype(np.float32)
    r[:, 3] = tmin
    r[:, 4:7] = dirs.astype(np.float32)
    r[:, 7] = tmax
    return r


def segment_rays(src, dst) -> np.ndarray:
    """Visibility segments src[i] -> dst[i]: d = dst - src (not normalised), t in (0, 1)."""
    src = np.asarray(src, dtype=np.float64)
    dst = np.asarray(dst, dtype=np.float64)
    r = np.empty((src.shape[0], 8), dtype=np.float32)
    r[:, 0:3] = src.astype(np.float32)
    r[:, 3] = 0.0
    r[:, 4:7] = (dst - src).astype(np.float32)
    r[:, 7] = 1.0
    return r


def random_rays(scene: Scene, n: int, seed: int, zmin=1.0, zmax=60.0, tmax=np.inf) -> np.ndarray:
    """Rays with origins uniform over the area at zmin..zmax m and uniform directions."""
    rng = _rng(seed)
    x0, y0, x1, y1 = scene.area
    o = np.stack([rng.uniform(x0, x1, n), rng.uniform(y0, y1, n), rng.uniform(zmin, zmax, n)], axis=1)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.empty((n, 8), dtype=np.float32)
    r[:, 0:3] = o.astype(np.float32)
    r[:, 3] = 0.0
    r[:, 4:7] = d.astype(np.float32)
    r[:, 7] = tmax
    return r


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------


def receiver_grid(size: float, k: int, z: float, x0: float = 0.0, y0: float = 0.0) -> np.ndarray:
    """k x k receivers at height z over the square [x0, x0 + size] x [y0, y0 + size],
    cell-centred, float32 [k * k, 3] (row-major in y, then x)."""
    c = (np.arange(k, dtype=np.float64) + 0.5) * (size / k)
    xx, yy = np.meshgrid(x0 + c, y0 + c)
    return np.stack([xx.ravel(), yy.ravel(), np.full(k * k, float(z))], 1).astype(np.float32)


def workload_tiny():
    """64-box city, 4096 Fibonacci rays from (100, 100, 30), t_max 1000 m, alpha 1."""
    sc = tiny_city(seed=1)
    rays = make_rays(sc.tx[0], fibonacci_directions(4096), 0.0, 1000.0)
    return sc, rays, dict(alpha=1.0, source=tuple(sc.tx[0]))


def workload_medium(level: int = 8):
    """1000-prism city, icosphere level-8 rays (655,362) from the centre at 30 m, t_max 500 m,
    in the launch order of the device generator (icosphere_launch_order)."""
    sc = medium_city(seed=2)
    rays = make_rays(sc.tx[0], icosphere_directions(level)[icosphere_launch_order(level)], 0.0, 500.0)
    return sc, rays, dict(alpha=0.4, source=tuple(sc.tx[0]))


def workload_batched(seed: int = 3):
    """10,000 convex 4-8-gon prisms on 3 x 3 km; 16 transmitters at 10-40 m with
    Fibonacci launches of log-uniform 64k-2M rays; a 64 x 64 receiver grid at 10 m."""
    rng = _rng(seed + 1000)
    size = 3000.0
    tx = np.stack([rng.uniform(0, size, 16), rng.uniform(0, size, 16), rng.uniform(10, 40, 16)], 1)
    counts = np.exp(rng.uniform(np.log(65536), np.log(2 * 1024 * 1024), 16)).astype(np.int64)
    sc = prism_city(10000, size, seed, tx_keepout=[tuple(t) for t in tx], name="batched_city")
    g = (np.arange(64) + 0.5) * (size / 64)
    gx, gy = np.meshgrid(g, g)
    rx = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 10.0)], 1)
    return sc, tx, counts, rx


def workload_large(seed: int = 5):
    """The large metro (about 13.2M triangles) with 32 transmitters, 2^21 Fibonacci rays
    each (67M rays, range 3 km), and 1M transmitter-receiver segments (32 x 32,768
    receivers).  Transmitters stand 10-40 m above the foot of 32 random building walls
    (so they follow the clustered buildings); receivers are uniform over the area at
    1.5-10 m."""
    sc = metro_city(seed=seed)
    rng = _rng(seed + 2000)
    walls = rng.integers(0, sc.n_tri - 2, 32)  # the last two triangles are the ground
    foot = sc.tris[walls].mean(axis=1)
    tx = np.stack([foot[:, 0], foot[:, 1], rng.uniform(10.0, 40.0, 32)], 1).astype(np.float32)
    counts = np.full(32, 1 << 21, np.int64)
    x0, y0, x1, y1 = sc.area
    n_rx = 32768
    rx = np.stack([rng.uniform(x0, x1, n_rx), rng.uniform(y0, y1, n_rx), rng.uniform(1.5, 10.0, n_rx)],
                  1).astype(np.float32)
    return sc, tx, counts, rx


def serving_scenes(n: int = 8, seed0: int = 101):
    """Resident scenes of 1000 .. 50000 buildings (log-spaced), generated as the
    1000-building city with other seeds; area grows with the building count."""
    counts = np.unique(np.round(np.exp(np.linspace(np.log(1000), np.log(50000), n))).astype(int))
    out = []
    for i, nb in enumerate(counts):
        size = 1000.0 * math.sqrt(nb / 1000.0)
        out.append(prism_city(int(nb), size, seed0 + i, name="serving_%d" % nb))
    return out


def serving_arrivals(scenes_, duration_s: float, rate_hz: float = 200.0, seed: int = 4):
    """Poisson arrivals: (time, scene index, tx, rays, max_order) with rays
    log-uniform 64k-4M and up to 2 reflections."""
    rng = _rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        k = int(rng.integers(0, len(scenes_)))
        x0, y0, x1, y1 = scenes_[k].area
        tx = (rng.uniform(x0, x1), rng.uniform(y0, y1), rng.uniform(10, 40))
        rays = int(np.exp(rng.uniform(np.log(65536), np.log(4 * 1024 * 1024))))
        out.append((t, k, tx, rays, int(rng.integers(0, 3))))
    return out
