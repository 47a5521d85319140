"""Band launch order of Fibonacci rays (no GPU): the library's slot -> direction
map equals a brute-force sort by azimuth, and the order makes each warp's 32
rays neighbours on the sphere."""
import ctypes

import numpy as np
import pytest

from paper_2208_10008_gb300 import rtbvh
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
    assert [lib.rt_launch_index(rtbvh.RT_RAYS_ICOSPHERE, 2, s) for s in (0, 5, 161)] == [0, 5, 161]
    assert rtbvh.rt_launch_index(rtbvh.RT_RAYS_FIBONACCI, 1, 0) == 0
