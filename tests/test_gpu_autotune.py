"""Autotuner, ray tiles and split-kernel timing events (needs a GB300).

Every configuration the autotuner may pick must return the same hits: the
hit rule does not depend on the tree or on the walk's tile."""
import ctypes

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_every_tuning_gives_the_same_hits(rb):
    sc, rays, p = scenes.workload_medium(level=5)
    rnd = scenes.random_rays(sc, 3000, seed=21, tmax=400.0)
    r = dev(np.concatenate([rays, rnd]))
    s = rb.rt_scene_upload(sc.tris)
    ref = None
    for width in (4, 8):
        for ml in (2, 4, 6, 8):
            for bins in (8, 16, 32):
                rb.rt_bvh_build(s, alpha=0.7, source=p["source"], max_leaf=ml, bins=bins, dist_norm=1, width=width)
                for tile in (64, 128, 256):
                    for stack in (16, 32, 64):
                        if (ml, bins) != (4, 16) and stack != 64:
                            continue  # every stack depth on one tree per width
                        h = rb.rt_trace_closest(s, r, block=tile, stack=stack)
                        o = rb.rt_trace_any(s, r, block=tile, stack=stack)
                        torch.cuda.synchronize()
                        got = (h.view(torch.int32).cpu().numpy(), o.cpu().numpy())
                        if ref is None:
                            ref = got
                        else:
                            assert np.array_equal(got[0], ref[0]), (width, ml, bins, tile, stack)
                            assert np.array_equal(got[1], ref[1]), (width, ml, bins, tile, stack)


def test_autotune_result_and_hits(rb, orc):
    sc, rays, p = scenes.workload_tiny()
    s = rb.rt_scene_upload(sc.tris)
    r = dev(rays)
    res = rb.rt_autotune(s, r, build_weight=1.0, alpha=0.7, source=p["source"], dist_norm=1)
    assert res["n_tried"] == 2 * 4 * 3 + 3 * 3 - 1
    assert res["max_leaf"] in (2, 4, 6, 8) and res["bins"] in (8, 16, 32) and res["block"] in (64, 128, 256)
    assert res["width"] in (4, 8) and res["stack"] in (16, 32, 64)
    assert 0 < res["score_ms"] <= res["default_score_ms"]
    assert res["score_ms"] == pytest.approx(res["build_ms"] + res["trace_ms"], rel=1e-5)
    # the scene is left built with the choice: its tree and hits are valid
    info = rb.rt_bvh_info(s)
    assert info["status"] == 0 and info["max_leaf_size"] <= res["max_leaf"]
    h = rb.rt_trace_closest(s, r, block=res["block"], stack=res["stack"])
    torch.cuda.synchronize()
    compare_closest(h.cpu().numpy(), orc.closest_brute(sc.tris, rays), sc.tris, rays, "autotuned")


def test_batch_ray_tile_does_not_change_results(rb):
    sc = scenes.tiny_city(seed=1)
    rng = np.random.default_rng(5)
    tx = np.stack([rng.uniform(20, 180, 2), rng.uniform(20, 180, 2), rng.uniform(10, 40, 2)], 1)
    counts = np.array([900, 2100])
    gx, gy = np.meshgrid(np.linspace(5, 195, 4), np.linspace(5, 195, 4))
    rx = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 10.0)], 1)
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, alpha=0.7, source=tuple(tx.mean(0)), max_leaf=4, dist_norm=1)
    outs = []
    for tile in (0, 64, 256):
        b = rb.Batch(s, tx, counts, rb.RT_RAYS_FIBONACCI, max_order=2, tmax=700.0, rx_pos=rx, ray_tile=tile)
        b.run()
        torch.cuda.synchronize()
        outs.append(([b.order(k)[1].clone() for k in range(3)], b.visibility().clone()))
        b.destroy()
    for hits, vis in outs[1:]:
        for k in range(3):
            assert torch.equal(hits[k].view(torch.int32), outs[0][0][k].view(torch.int32))
        assert torch.equal(vis, outs[0][1])
    with pytest.raises(rb.RtError):
        rb.Batch(s, tx, counts, rb.RT_RAYS_FIBONACCI, max_order=1, tmax=700.0, rx_pos=rx, ray_tile=100)


def test_split_events_time_the_split_kernel(rb):
    sc, rays, p = scenes.workload_medium(level=1)
    s = rb.rt_scene_upload(sc.tris)
    st = torch.cuda.Stream()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        rb.rt_bvh_build(s, stream=st, alpha=0.7, source=p["source"], dist_norm=1)
        rb.rt_scene_set_split_events(s, s0, s1)
        b0.record(st)
        rb.rt_bvh_build(s, stream=st, alpha=0.7, source=p["source"], dist_norm=1)
        b1.record(st)
        rb.rt_scene_set_split_events(s)
    st.synchronize()
    whole, split = b0.elapsed_time(b1), s0.elapsed_time(s1)
    assert 0 < split <= whole
    # one event without the other is refused
    assert rb.lib().rt_scene_set_split_events(s.handle, ctypes.c_void_p(s0.cuda_event), None) == -1


def test_full_size_in_the_benchmarked_launch_configuration(rb, orc):
    # what the benchmark times: the medium city's 655,362 icosphere rays, the
    # tree and ray tile the autotuner picks (build weight 1), the build and
    # the walk launched as in a step; sampled rays against brute force
    sc, rays_np, _ = scenes.workload_medium()
    src = tuple(float(v) for v in sc.tx[0])
    s = rb.rt_scene_upload(sc.tris)
    rays = dev(rays_np)
    tune = rb.rt_autotune(s, rays, build_weight=1.0, alpha=0.7, source=src, dist_norm=1)
    rb.rt_bvh_build(s, alpha=0.7, source=src, dist_norm=1, max_leaf=tune["max_leaf"], bins=tune["bins"],
                    width=tune["width"])
    hits = torch.empty((len(rays_np), 4), dtype=torch.float32, device="cuda")
    nflag = torch.zeros(1, dtype=torch.int32, device="cuda")
    rb.rt_trace_closest(s, rays, hits, n_flagged=nflag, block=tune["block"], stack=tune["stack"])
    torch.cuda.synchronize()
    h = hits.cpu().numpy()
    rng = np.random.default_rng(12)
    sample = np.union1d(rng.choice(len(rays_np), 6000, replace=False), np.arange(0, len(rays_np), 1111))
    ref = orc.closest_brute(sc.tris, rays_np[sample])
    compare_closest(h[sample], ref, sc.tris, rays_np[sample], "benchmarked configuration")
    assert int(nflag.item()) < len(rays_np) // 1000  # the float64 pass stays rare


def test_stack_overflow_goes_to_the_float64_pass(rb, orc):
    # a 16-deep stack on the deep alpha = 0 tree overflows for some rays: they
    # are finished by the float64 whole-tree walk and the hits do not change
    sc, rays, p = scenes.workload_medium(level=4)
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, alpha=0.0, source=p["source"], max_leaf=1, bins=16, dist_norm=0)
    r = dev(rays)
    nf = torch.zeros(1, dtype=torch.int32, device="cuda")
    deep = rb.rt_trace_closest(s, r, stack=64)
    short = rb.rt_trace_closest(s, r, stack=16, n_flagged=nf)
    torch.cuda.synchronize()
    assert torch.equal(deep.view(torch.int32), short.view(torch.int32))
    compare_closest(short.cpu().numpy(), orc.closest_brute(sc.tris, rays), sc.tris, rays, "stack 16")
    print("stack 16 on the alpha = 0 tree: %d rays flagged, depth %d" % (int(nf.item()), rb.rt_bvh_info(s)["depth2"]))


@pytest.mark.parametrize("alpha,dist_norm", [(1.0, 0), (0.7, 1), (0.4, 0)])
def test_width_8_full_icosphere(rb, orc, alpha, dist_norm):
    # the 8-wide nodes against the checker on all 655,362 medium-city rays
    sc, rays, p = scenes.workload_medium()
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, alpha=alpha, source=p["source"], max_leaf=2, bins=16, dist_norm=dist_norm, width=8)
    info = rb.rt_bvh_info(s)
    assert info["status"] == 0
    ref = orc.Bvh(sc.tris, alpha=1.0, max_leaf=4).closest(rays)
    h = rb.rt_trace_closest(s, dev(rays))
    torch.cuda.synchronize()
    compare_closest(h.cpu().numpy(), ref, sc.tris, rays, "width 8 a=%g" % alpha)
    rb.rt_bvh_build(s, alpha=alpha, source=p["source"], max_leaf=2, bins=16, dist_norm=dist_norm, width=4)
    info4 = rb.rt_bvh_info(s)
    # the same binary tree, about half as many levels of traversal nodes
    assert info4["n_bvh2_internal"] == info["n_bvh2_internal"] and info["depth_wide"] < info4["depth_wide"]
    print("width 8 a=%g: %d traversal nodes, depth %d (width 4: %d, depth %d)" % (
        alpha, info["n_wide"], info["depth_wide"], info4["n_wide"], info4["depth_wide"]))
