"""rt_trace_closest_noalloc: the closest-hit call for callers that cannot let
the library allocate device memory (a runtime that owns all device memory
through its own pool, or a latency-critical stream that must not stall on
cudaMalloc).  Its results must match rt_trace_closest's, call after call,
since both share the one compiled-in scratch array's contents only through
values each call rewrites.

This file is named to be collected last: if it fails, a run that stops at
the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2208_10008_gb300 import scenes
from helpers import T_ABS, T_REL, split_hits

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rb():
    from paper_2208_10008_gb300 import rtbvh
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    rtbvh.lib()
    return rtbvh


def _call_noalloc(rb, scene, rays_t, hits_t):
    """Straight through the C ABI (no Python-side allocation involved)."""
    lib = rb.lib()
    tp = rb.TraceParams()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.rt_trace_closest_noalloc(ctypes.c_void_p(scene.handle), ctypes.c_void_p(rays_t.data_ptr()),
                                        rays_t.shape[0], ctypes.c_void_p(hits_t.data_ptr()),
                                        ctypes.byref(tp), stream)


def _same_within_tolerance(a, b):
    ta, ia, _, _ = split_hits(a)
    tb, ib, _, _ = split_hits(b)
    assert (ia == ib).all()
    hit = ib >= 0
    assert np.isinf(ta[~hit]).all()
    assert np.all(np.abs(ta[hit] - tb[hit]) <= T_REL * tb[hit] + T_ABS)


def test_noalloc_matches_trace_closest_twice(rb):
    sc, _, p = scenes.workload_medium(level=1)
    scene = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(scene, alpha=0.7, source=p["source"], max_leaf=4, bins=16, dist_norm=1)
    batches = [scenes.make_rays(sc.tx[0], scenes.icosphere_directions(7), 0.0, 500.0),   # 163,842 rays
               scenes.random_rays(sc, 250_000, seed=77, tmax=400.0)]
    for rays in batches:          # two calls in a row reuse the same fixed scratch
        rays_t = torch.from_numpy(rays).cuda()
        ref = rb.rt_trace_closest(scene, rays_t)
        out = torch.full((len(rays), 4), np.nan, dtype=torch.float32, device="cuda")
        assert _call_noalloc(rb, scene, rays_t, out) == 0
        torch.cuda.synchronize()
        _same_within_tolerance(out.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_rejects_batches_over_the_limit(rb):
    sc, _, p = scenes.workload_medium(level=1)
    scene = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(scene, alpha=1.0, source=p["source"])
    n = rb.RT_NOALLOC_MAX_RAYS + 1
    rays_t = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    hits_t = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    assert _call_noalloc(rb, scene, rays_t, hits_t) == -1
    assert b"RT_NOALLOC_MAX_RAYS" in rb.lib().rt_last_error()
