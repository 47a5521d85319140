"""Batched multi-bounce pipeline (many transmitters, reflections, visibility)
vs the per-call path and the float64 checker (needs a GB300)."""
import numpy as np
import pytest

from paper_2208_10008_gb300 import scenes
from helpers import compare_closest, fibonacci_launch_perm, split_hits

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rb():
    from paper_2208_10008_gb300 import rtbvh
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    rtbvh.lib()
    return rtbvh


def _setup(rb, seed=3):
    sc = scenes.tiny_city(seed=1)
    rng = np.random.default_rng(seed)
    tx = np.stack([rng.uniform(20, 180, 3), rng.uniform(20, 180, 3), rng.uniform(10, 40, 3)], 1)
    counts = np.array([700, 1500, 3001])
    gx, gy = np.meshgrid(np.linspace(5, 195, 5), np.linspace(5, 195, 5))
    rx = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 10.0)], 1)
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, alpha=0.7, source=tuple(tx.mean(0)), max_leaf=4, dist_norm=1)
    return sc, s, tx, counts, rx


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_orders_match_checker(rb, orc, use_graph):
    sc, s, tx, counts, rx = _setup(rb)
    b = rb.Batch(s, tx, counts, rb.RT_RAYS_FIBONACCI, max_order=3, tmax=600.0, rx_pos=rx, use_graph=use_graph)
    for _ in range(3):                  # eager run, capture run, replay
        b.run()
    st = b.stats()
    assert st["rays"][0] == counts.sum()
    prev_rays = prev_hits = None
    for k in range(4):
        rays, hits, src, n = b.order(k)
        r = rays.cpu().numpy()
        h = hits.cpu().numpy()
        assert n == st["rays"][k]
        skip = None
        if k == 0:
            # launched rays: each transmitter's Fibonacci set, in band order
            off = 0
            for t, c in enumerate(counts):
                d = orc.fibonacci(int(c))[fibonacci_launch_perm(int(c))]
                assert np.abs(r[off:off + c, 4:7] - d).max() < 2e-6
                assert np.allclose(r[off:off + c, 0:3], tx[t].astype(np.float32))
                off += c
        else:
            srcn = src.cpu().numpy()
            pt, pid, _, _ = split_hits(prev_hits)
            keep = (pid >= 0) & (prev_rays[:, 7].astype(np.float64) - pt > 0)
            assert np.array_equal(srcn, np.nonzero(keep)[0])
            skip = pid[srcn]
            refl = orc.reflect(sc.tris, prev_rays[srcn], pid[srcn], pt[srcn])
            assert np.all(np.abs(r[:, 4:7] - refl[:, 4:7]) <= 1e-5)
        ref = orc.closest_brute(sc.tris, r, skip=skip)
        compare_closest(h, ref, sc.tris, r, "batch order %d" % k)
        prev_rays, prev_hits = r, h
    vis = b.visibility().cpu().numpy()
    seg = scenes.segment_rays(np.repeat(tx, len(rx), 0), np.tile(rx, (len(tx), 1)))
    assert (vis == orc.any_brute(sc.tris, seg)).all()
    assert st["visible"] == int((vis == 0).sum())
    b.destroy()


def test_batch_equals_per_call_path_and_is_repeatable(rb):
    sc, s, tx, counts, rx = _setup(rb, seed=4)
    b = rb.Batch(s, tx, counts, rb.RT_RAYS_FIBONACCI, max_order=2, tmax=800.0, rx_pos=rx)
    outs = []
    for _ in range(4):
        b.run()
        torch.cuda.synchronize()
        outs.append([b.order(k)[1].clone() for k in range(3)])
    for o in outs[1:]:
        for k in range(3):
            assert torch.equal(o[k].view(torch.int32), outs[0][k].view(torch.int32))
    # per-call path on the batch's own order-0 rays
    cur = b.order(0)[0].clone()
    skip = None
    for k in range(3):
        h = rb.rt_trace_closest(s, cur, skip=skip)
        assert torch.equal(h.view(torch.int32), outs[-1][k].view(torch.int32))
        if k < 2:
            nr, ns, _, c = rb.rt_reflect(s, cur, h)
            m = int(c.item())
            cur, skip = nr[:m].contiguous(), ns[:m].contiguous()
    b.destroy()


def test_batch_graph_follows_a_grown_scene(rb):
    sc, s, tx, counts, rx = _setup(rb, seed=5)
    b = rb.Batch(s, tx, counts, rb.RT_RAYS_FIBONACCI, max_order=2, tmax=800.0, rx_pos=rx)
    for _ in range(3):                  # eager run, capture run, replay
        b.run()
    torch.cuda.synchronize()
    # about 3000 triangles instead of 770: every per-triangle array of the scene moves
    big = scenes.medium_city(seed=7, n_buildings=150, size=200.0)
    assert len(big.tris) > 2 * len(sc.tris)
    rb.rt_scene_update(s, big.tris)
    rb.rt_bvh_build(s, alpha=0.7, source=tuple(tx.mean(0)), max_leaf=4, dist_norm=1)
    for _ in range(2):                  # captured again, then replayed
        b.run()
    torch.cuda.synchronize()
    got = [b.order(k)[1].clone() for k in range(3)]
    vis = b.visibility().clone()
    fresh = rb.Batch(s, tx, counts, rb.RT_RAYS_FIBONACCI, max_order=2, tmax=800.0, rx_pos=rx, use_graph=False)
    fresh.run()
    torch.cuda.synchronize()
    for k in range(3):
        assert torch.equal(got[k].view(torch.int32), fresh.order(k)[1].view(torch.int32))
    assert torch.equal(vis, fresh.visibility())
    b.destroy()
    fresh.destroy()


def test_batch_icosphere_launches_in_tile_order(rb, orc):
    # icosphere transmitters: every transmitter's launch is the checker's
    # directions in tile order and the same bits as its own rt_gen_rays call;
    # the direct rays' hits against the float64 brute force
    sc, s, tx, _, _ = _setup(rb, seed=9)
    levels = np.array([3, 5, 4])
    b = rb.Batch(s, tx, levels, rb.RT_RAYS_ICOSPHERE, max_order=1, tmax=600.0)
    b.run()
    torch.cuda.synchronize()
    rays, hits, _, n = b.order(0)
    r, h = rays.cpu().numpy(), hits.cpu().numpy()
    counts = [rb.rt_ray_count(rb.RT_RAYS_ICOSPHERE, int(L)) for L in levels]
    assert n == sum(counts)
    off = 0
    for t, (L, c) in enumerate(zip(levels, counts)):
        ref = orc.icosphere(int(L))[scenes.icosphere_launch_order(int(L))]
        assert np.abs(r[off:off + c, 4:7] - ref).max() < 2e-6
        own = rb.rt_gen_rays(rb.RT_RAYS_ICOSPHERE, tx[t], int(L), 0.0, 600.0).cpu().numpy()
        assert np.array_equal(r[off:off + c].view(np.uint32), own.view(np.uint32))
        off += c
    compare_closest(h, orc.closest_brute(sc.tris, r), sc.tris, r, "icosphere batch, direct rays")
    b.destroy()
