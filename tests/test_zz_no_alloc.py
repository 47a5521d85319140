"""rt_trace_closest_noalloc: the closest-hit call for callers that cannot let
the library allocate device memory (a runtime that owns all device memory
through its own pool, or a latency-critical stream that must not stall on
cudaMalloc).  It runs the same kernels on the same tree as rt_trace_closest,
so its hit records must equal rt_trace_closest's bit for bit, call after
call, even though every call reuses the one compiled-in scratch array.

This file is named to be collected last: if it fails, a run that stops at
the first failure has already run every other test.
"""
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


def _call_noalloc(rb, scene, rays_t, hits_t, n_flagged_t=None):
    """Straight through the C ABI (no Python-side allocation involved)."""
    lib = rb.lib()
    tp = rb.TraceParams()
    if n_flagged_t is not None:
        tp.n_flagged_dev = n_flagged_t.data_ptr()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.rt_trace_closest_noalloc(ctypes.c_void_p(scene.handle), ctypes.c_void_p(rays_t.data_ptr()),
                                        rays_t.shape[0], ctypes.c_void_p(hits_t.data_ptr()),
                                        ctypes.byref(tp), stream)


def _vertex_rays(sc, k, seed):
    """Rays from the transmitter straight at k triangle vertices: each passes
    through a corner that several facets share, which the float32 pass cannot
    settle, so these rays go through the float64 re-test queue."""
    rng = np.random.default_rng(seed)
    pick = rng.integers(0, sc.n_tri - 2, k)
    v = sc.tris[pick, rng.integers(0, 3, k)].astype(np.float64)
    d = v - sc.tx[0]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return scenes.make_rays(sc.tx[0], d, 0.0, 500.0)


def test_noalloc_first_on_a_fresh_scene_then_bit_equal_twice(rb, orc):
    sc, _, p = scenes.workload_medium(level=1)
    # set-up of the fixed array on this device (its first call) on a scene of its own
    warm = rb.rt_scene_upload(sc.tris[:100].copy())
    rb.rt_bvh_build(warm)
    w_rays = torch.from_numpy(_vertex_rays(sc, 64, 1)).cuda()
    w_hits = torch.empty((64, 4), dtype=torch.float32, device="cuda")
    assert _call_noalloc(rb, warm, w_rays, w_hits) == 0
    torch.cuda.synchronize()

    scene = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(scene, alpha=0.7, source=p["source"], max_leaf=4, bins=16, dist_norm=1)
    batches = [np.concatenate([scenes.make_rays(sc.tx[0], scenes.icosphere_directions(7), 0.0, 500.0),
                               _vertex_rays(sc, 2000, 2)]),                       # 165,842 rays
               scenes.random_rays(sc, 250_000, seed=77, tmax=400.0)]
    for b, rays in enumerate(batches):   # two calls in a row reuse the same fixed scratch
        rays_t = torch.from_numpy(rays).cuda()
        out = torch.full((len(rays), 4), np.nan, dtype=torch.float32, device="cuda")
        nf = torch.zeros(1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        # on the fresh scene, before any rt_trace_closest could have grown its scratch
        assert _call_noalloc(rb, scene, rays_t, out, nf) == 0
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        # rt_trace_closest would grow the scene's re-test scratch by 40 B per ray here
        # (6.6 MB for this batch); this call takes nothing from the device
        assert free0 - free1 < 2 * 1024 * 1024, (free0, free1)
        n_flagged = int(nf.item())
        if b == 0:
            assert n_flagged >= 100, n_flagged   # the re-test queue in the fixed array was used
        ref = rb.rt_trace_closest(scene, rays_t)
        torch.cuda.synchronize()
        a, r = out.cpu().numpy(), ref.cpu().numpy()
        assert np.array_equal(a.view(np.uint32), r.view(np.uint32)), "batch %d differs from rt_trace_closest" % b
        # and a sample (with every vertex ray of the first batch) against the float64 brute force
        k = np.random.default_rng(b).choice(len(rays), 3000, replace=False)
        if b == 0:
            k = np.unique(np.concatenate([k, np.arange(len(rays) - 2000, len(rays))]))
        compare_closest(a[k], orc.closest_brute(sc.tris, rays[k]), sc.tris, rays[k], "noalloc batch %d" % b)
        print("noalloc batch %d: %d rays, %d flagged, free memory %d -> %d" % (b, len(rays), n_flagged, free0,
                                                                           free1))


def test_noalloc_rejects_batches_over_the_limit(rb):
    sc, _, p = scenes.workload_medium(level=1)
    scene = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(scene, alpha=1.0, source=p["source"])
    n = rb.RT_NOALLOC_MAX_RAYS + 1
    rays_t = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    hits_t = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    assert _call_noalloc(rb, scene, rays_t, hits_t) == -1
    assert b"RT_NOALLOC_MAX_RAYS" in rb.lib().rt_last_error()
