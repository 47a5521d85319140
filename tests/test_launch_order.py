"""Launch orders (no GPU): the library's slot -> direction map equals, for
Fibonacci rays, a brute-force sort of each band by azimuth and, for icosphere
rays, the host generator's tile order; both make each warp's 32 rays
neighbours on the sphere."""
import ctypes

import numpy as np
import pytest

from paper_2208_10008_gb300 import rtbvh, scenes
from helpers import fibonacci_launch_perm


def _band_width(n):
    a, w = 1, 2
    while (a + w) ** 2 <= 80 * n:
        a, w = w, a + w
    return w, a + w


@pytest.mark.parametrize("n", [1, 7, 64, 700, 4096, 65536, 1_000_000])
def test_perm_is_banded_azimuth_order(orc, n):
    perm = fibonacci_launch_perm(n)
    assert np.array_equal(np.sort(perm), np.arange(n))
    w, w_next = _band_width(n)
    assert w * w <= 80 * n < w_next * w_next
    full = (n // w) * w
    assert np.array_equal(perm[full:], np.arange(full, n))           # the tail keeps spiral order
    if full == 0:
        return
    d = orc.fibonacci(n)
    az = np.arctan2(d[:, 1], d[:, 0])
    for b in range(n // w):
        seg = perm[b * w:(b + 1) * w]
        assert seg[0] == b * w and np.array_equal(np.sort(seg), np.arange(b * w, (b + 1) * w))
        # azimuth measured from the band's first point rises along the slots
        rel = np.mod(az[seg] - az[b * w], 2 * np.pi)
        assert (np.diff(rel) > 0).all()


def _warp_spread(d):
    m = (d.shape[0] // 32) * 32
    x = d[:m].reshape(-1, 32, 3)
    c = x.mean(1)
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    return np.median(np.arccos(np.clip((x * c[:, None, :]).sum(2), -1, 1)).max(1))


@pytest.mark.parametrize("n", [65536, 1 << 21])
def test_band_order_makes_warps_coherent(orc, n):
    d = orc.fibonacci(n)
    spiral = _warp_spread(d)
    band = _warp_spread(d[fibonacci_launch_perm(n)])
    # a warp of spiral-order rays spans about a radian of azimuth; in band
    # order it covers a patch of 32 rays: a disc of 32 ray cells has a radius
    # of sqrt(32 / pi) = 3.2 mean spacings
    spacing = np.sqrt(4 * np.pi / n)
    assert spiral > 1.0
    assert band < 6.0 * spacing


@pytest.mark.parametrize("n", [1, 7, 64, 700, 4096, 65536, 1_000_000])
def test_library_launch_index_matches_brute_force_without_gpu(n):
    lib = rtbvh.lib()
    perm = fibonacci_launch_perm(n)
    slots = np.arange(n) if n <= 70000 else np.unique(np.r_[np.arange(0, n, 97), np.arange(n - 7000, n)])
    got = np.array([lib.rt_launch_index(rtbvh.RT_RAYS_FIBONACCI, n, int(s)) for s in slots], dtype=np.int64)
    assert np.array_equal(got, perm[slots])


def test_launch_index_edges_without_gpu():
    lib = rtbvh.lib()
    assert lib.rt_launch_index(rtbvh.RT_RAYS_FIBONACCI, 100, -1) == -1
    assert lib.rt_launch_index(rtbvh.RT_RAYS_FIBONACCI, 100, 100) == -1
    assert lib.rt_launch_index(rtbvh.RT_RAYS_FIBONACCI, 0, 0) == -1
    assert lib.rt_launch_index(7, 100, 3) == -1
    assert lib.rt_launch_index(rtbvh.RT_RAYS_ICOSPHERE, 13, 0) == -1
    assert lib.rt_launch_index(rtbvh.RT_RAYS_ICOSPHERE, 2, 162) == -1
    # level 2: every face holds 3 points in rows 1 and 2 (no full band): the identity
    assert [lib.rt_launch_index(rtbvh.RT_RAYS_ICOSPHERE, 2, s) for s in range(162)] == list(range(162))
    assert rtbvh.rt_launch_index(rtbvh.RT_RAYS_FIBONACCI, 1, 0) == 0


@pytest.mark.parametrize("level", range(0, 9))
def test_library_icosphere_order_matches_host_without_gpu(level):
    lib = rtbvh.lib()
    perm = scenes.icosphere_launch_order(level)
    n = len(perm)
    assert n == 10 * 4 ** level + 2 and np.array_equal(np.sort(perm), np.arange(n))
    slots = np.arange(n) if n <= 200_000 else np.unique(np.r_[np.arange(0, n, 7), np.arange(n - 5000, n)])
    got = np.array([lib.rt_launch_index(rtbvh.RT_RAYS_ICOSPHERE, level, int(s)) for s in slots], dtype=np.int64)
    assert np.array_equal(got, perm[slots])


def _face_point(level, k):
    """(face, row i, column j) of a face point given by its icosphere_directions index."""
    f = 1 << level
    q = k - 12 - 30 * (f - 1)
    per_face = (f - 1) * (f - 2) // 2
    fc, q = divmod(q, per_face)
    i = 1
    while q >= f - 1 - i:
        q -= f - 1 - i
        i += 1
    return fc, i, q + 1


def test_icosphere_tiles_are_8_by_4_lattice_blocks():
    # level 6 (f = 64): the first band of face 0 starts with its tiles, each
    # 32 slots covering rows 1..8 and 4 adjacent columns; band 1 (rows 9..16)
    # starts with its rest and ends with its first tile
    level, f = 6, 64
    perm = scenes.icosphere_launch_order(level)
    head = 12 + 30 * (f - 1)
    for t in range(3):
        pts = [_face_point(level, int(perm[head + 32 * t + u])) for u in range(32)]
        assert {p[0] for p in pts} == {0}
        assert sorted({p[1] for p in pts}) == list(range(1, 9))
        assert sorted({p[2] for p in pts}) == [4 * t + 1 + c for c in range(4)]
    band0 = 8 * (f - 2) - 28
    first_of_band1 = _face_point(level, int(perm[head + band0]))
    last_of_band1 = _face_point(level, int(perm[head + band0 + 8 * (f - 10) - 28 - 1]))
    assert first_of_band1[1] == 9 and first_of_band1[2] > 40      # the rest lies at the far end
    assert last_of_band1[1] == 16 and last_of_band1[2] == 4        # the first tile ends the band


def test_icosphere_tile_order_makes_warps_coherent():
    d = scenes.icosphere_directions(8)
    spacing = np.sqrt(4 * np.pi / len(d))
    assert _warp_spread(d) > 10 * spacing                # rows of 32 points along a face, edges
    assert _warp_spread(d[scenes.icosphere_launch_order(8)]) < 6 * spacing


@pytest.mark.parametrize("level", [10, 12])
def test_library_icosphere_order_high_levels_sampled_without_gpu(level):
    lib = rtbvh.lib()
    perm = scenes.icosphere_launch_order(level)
    n = len(perm)
    rng = np.random.default_rng(level)
    f = 1 << level
    head = 12 + 30 * (f - 1)
    per_face = (f - 1) * (f - 2) // 2
    slots = np.unique(np.r_[rng.integers(0, n, 20000), np.arange(head, head + 3000),
                            np.arange(n - per_face - 1000, n - per_face + 1000), np.arange(n - 3000, n)])
    got = np.array([lib.rt_launch_index(rtbvh.RT_RAYS_ICOSPHERE, level, int(s)) for s in slots], dtype=np.int64)
    assert np.array_equal(got, perm[slots])


def test_library_launch_index_many_counts_without_gpu():
    # 52 distinct seeded ray counts from 1 to 3M, which meet every band width
    # from 8 to 10,946 (both parities of the step rule): sampled slots of each
    # against the brute-force azimuth sort
    lib = rtbvh.lib()
    rng = np.random.default_rng(2208)
    counts = np.unique(np.r_[np.exp(rng.uniform(0, np.log(3e6), 58)).astype(np.int64), 1, 3_000_000])
    for n in counts:
        n = int(n)
        perm = fibonacci_launch_perm(n)
        k = np.unique(np.r_[rng.integers(0, n, 300), np.arange(max(0, n - 40), n)])
        got = np.array([lib.rt_launch_index(rtbvh.RT_RAYS_FIBONACCI, n, int(s)) for s in k], dtype=np.int64)
        assert np.array_equal(got, perm[k]), n
