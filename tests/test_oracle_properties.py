"""Randomised properties of the float64 checker (no GPU; needs hypothesis,
skipped where it is not installed): over many seeded small scenes and ray
sets, the exact-sweep BVH walk of Sec. II.C / Fig. 4 equals brute force bit
for bit at every alpha, distance variant and leaf size, and any-hit equals
"closest t < tmax"."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


def _scene(rng, n):
    # clustered small triangles plus a few large ones, some degenerate
    c = rng.uniform(-20, 20, (n, 1, 3))
    t = (c + rng.normal(0, 3, (n, 3, 3))).astype(np.float32)
    k = rng.integers(0, n, max(1, n // 10))
    t[k, 2] = t[k, 1]  # a repeated vertex: zero area
    return t


def _rays(rng, m):
    o = rng.uniform(-30, 30, (m, 3))
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tmin = np.where(rng.random(m) < 0.2, rng.uniform(0, 5, m), 0.0)
    tmax = np.where(rng.random(m) < 0.5, rng.uniform(5, 60, m), np.inf)
    return np.concatenate([o, tmin[:, None], d, tmax[:, None]], 1).astype(np.float32)


@settings(max_examples=40, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), n=st.integers(1, 60), alpha=st.sampled_from([0.0, 0.4, 0.7, 1.0]),
       max_leaf=st.integers(1, 8), dist_norm=st.integers(0, 1))
def test_bvh_walk_equals_brute_force(orc, seed, n, alpha, max_leaf, dist_norm):
    rng = np.random.default_rng(seed)
    tris = _scene(rng, n)
    rays = _rays(rng, 200)
    src = tuple(rng.uniform(-20, 20, 3))
    bvh = orc.Bvh(tris, alpha=alpha, source=src, max_leaf=max_leaf, dist_norm=dist_norm)
    a = orc.closest_brute(tris, rays)
    b = bvh.closest(rays)
    assert np.array_equal(a.id, b.id)
    assert np.array_equal(a.t, b.t)
    inf = bvh.info()
    assert inf["largest_leaf"] <= max_leaf and inf["prims"] == n


@settings(max_examples=30, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), n=st.integers(1, 60))
def test_any_hit_is_closest_within_range(orc, seed, n):
    rng = np.random.default_rng(seed)
    tris = _scene(rng, n)
    rays = _rays(rng, 300)
    h = orc.closest_brute(tris, rays)
    anyh = orc.any_brute(tris, rays)
    assert np.array_equal(anyh.astype(bool), h.id >= 0)
