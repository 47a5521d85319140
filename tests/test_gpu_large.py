"""The large metro at full size (about 13.2 million triangles; needs a
GB300): build with the Eq. 2 cost, check the tree's counts, and compare
seeded samples with the float64 brute force: 16,384 transmitter rays, 4,096
random rays and 16,384 of the 1M transmitter-receiver visibility segments.

The brute force of a group of rays runs over the triangles whose box lies
within the group's reach (for rays from one point: the ball of radius
tmax |d| around it; for rays from a cell: that cell grown by tmax |d|).
That leaves the answer unchanged: a hit at t < tmax lies inside the reach,
and so does the box of its triangle.  The triangles keep their order, so
ties still go to the lowest id."""
import numpy as np
import pytest

from paper_2208_10008_gb300 import scenes
from helpers import compare_closest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rb():
    from paper_2208_10008_gb300 import rtbvh
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    rtbvh.lib()
    return rtbvh


@pytest.fixture(scope="module")
def metro(rb):
    sc, tx, counts, rx = scenes.workload_large()
    assert sc.n_tri > 13_000_000
    s = rb.rt_scene_upload(sc.tris)
    centre = (10_000.0, 10_000.0, 30.0)
    rb.rt_bvh_build(s, alpha=0.7, source=centre, max_leaf=4, bins=16, dist_norm=1)
    rb.rt_bvh_build(s, alpha=0.7, source=centre, max_leaf=4, bins=16, dist_norm=1)  # timed (buffers exist)
    lo = sc.tris.min(axis=1)
    hi = sc.tris.max(axis=1)
    yield sc, tx, counts, rx, s, lo, hi
    s.destroy()


def _within(lo, hi, blo, bhi, reach):
    """Triangles whose box comes within `reach` of the box [blo, bhi] (per-axis gap test)."""
    gap = np.maximum(np.maximum(blo[None, :] - hi, lo - bhi[None, :]), 0.0)
    return np.nonzero((gap.astype(np.float64) ** 2).sum(1) <= reach * reach)[0]


def _closest_pruned(orc, tris, lo, hi, rays, blo, bhi, reach):
    keep = _within(lo, hi, blo, bhi, reach)
    ref = orc.closest_brute(tris[keep], rays)
    hit = ref.id >= 0
    ref.id[hit] = keep[ref.id[hit]].astype(np.int32)
    return ref, len(keep)


def test_metro_build(rb, metro):
    sc, tx, counts, rx, s, lo, hi = metro
    info = rb.rt_bvh_info(s)
    print("metro: %d triangles, build %.2f ms, depth %d, %d traversal nodes" % (
        info["n_tri"], info["build_ms"], info["depth2"], info["n_wide"]))
    assert info["status"] == 0 and info["n_tri"] == sc.n_tri
    assert info["n_leaves"] == info["n_bvh2_internal"] + 1 and info["max_leaf_size"] <= 4


def test_metro_transmitter_rays(rb, orc, metro):
    # 4 of the 32 transmitters, 2^21 Fibonacci rays each (range 3 km) as the
    # benchmark launches them; 4,096 seeded rays of each against brute force
    sc, tx, counts, rx, s, lo, hi = metro
    rng = np.random.default_rng(71)
    tmax = 3000.0
    for t in range(4):
        rays_d = rb.rt_gen_rays(rb.RT_RAYS_FIBONACCI, tx[t], int(counts[t]), 0.0, tmax)
        h = rb.rt_trace_closest(s, rays_d)
        o = rb.rt_trace_any(s, rays_d)
        torch.cuda.synchronize()
        hits, occl = h.cpu().numpy(), o.cpu().numpy()
        ids = hits[:, 1].view(np.int32)
        assert np.array_equal(occl != 0, ids >= 0)  # any-hit == closest t < tmax, every ray
        k = np.sort(rng.choice(len(hits), 4096, replace=False))
        rays = rays_d[torch.from_numpy(k).cuda()].cpu().numpy()
        p = np.asarray(tx[t], np.float32)
        ref, nkept = _closest_pruned(orc, sc.tris, lo, hi, rays, p, p, tmax * 1.0001 + 1.0)
        n, nh, nt = compare_closest(hits[k], ref, sc.tris, rays, "metro tx %d" % t)
        print("metro tx %d: %d rays, %d hits, %d near-ties, %d triangles within reach" % (t, n, nh, nt, nkept))


def test_metro_random_rays(rb, orc, metro):
    # random origins and directions over the whole metro (range 2 km), checked
    # in 4 x 4 km cells of origins
    sc, tx, counts, rx, s, lo, hi = metro
    tmax = 2000.0
    rays = scenes.random_rays(sc, 4096, seed=56, tmax=tmax)
    h = rb.rt_trace_closest(s, torch.from_numpy(rays).cuda())
    torch.cuda.synchronize()
    hits = h.cpu().numpy()
    cell = 4000.0
    key = np.floor(rays[:, 0] / cell).astype(np.int64) * 100 + np.floor(rays[:, 1] / cell).astype(np.int64)
    for c in np.unique(key):
        m = np.nonzero(key == c)[0]
        blo = rays[m, :3].min(0)
        bhi = rays[m, :3].max(0)
        reach = tmax * float(np.linalg.norm(rays[m, 4:7], axis=1).max()) * 1.0001 + 1.0
        ref, _ = _closest_pruned(orc, sc.tris, lo, hi, rays[m], blo, bhi, reach)
        compare_closest(hits[m], ref, sc.tris, rays[m], "metro random cell %d" % c)


def test_metro_visibility_pairs(rb, orc, metro):
    # the 1M transmitter-receiver segments of the benchmark (32 x 32,768);
    # a seeded 16,384 of them against the float64 any-hit brute force
    sc, tx, counts, rx, s, lo, hi = metro
    seg = scenes.segment_rays(np.repeat(tx, len(rx), 0), np.tile(rx, (len(tx), 1)))
    occ = rb.rt_trace_any(s, torch.from_numpy(seg).cuda())
    torch.cuda.synchronize()
    occ = occ.cpu().numpy()
    k = np.sort(np.random.default_rng(72).choice(len(seg), 16384, replace=False))
    ref = orc.any_brute(sc.tris, seg[k])
    assert np.array_equal(occ[k], ref), "%d of %d segments differ" % (int((occ[k] != ref).sum()), len(k))
    print("metro visibility: %d of %d segments visible (sample: %d of %d)" % (
        int((occ == 0).sum()), len(seg), int((ref == 0).sum()), len(k)))
