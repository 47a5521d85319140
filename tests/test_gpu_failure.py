"""Failure detection without a GPU fault (needs a GB300).

Waits of the build run out on purpose (pending work that is never
published, through the test hooks), allocations fail on purpose; each time
the call reports the error and the context stays usable."""
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
    yield rtbvh
    for hook in (1, 2, 3, 4):
        rtbvh.rt_debug_inject(hook, 0)


def _check_usable(rb, orc):
    sc, rays, p = scenes.workload_tiny()
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, source=p["source"])
    assert rb.rt_bvh_info(s)["status"] == 0
    h = rb.rt_trace_closest(s, torch.from_numpy(rays).cuda())
    torch.cuda.synchronize()
    compare_closest(h.cpu().numpy(), orc.closest_brute(sc.tris, rays), sc.tris, rays, "after failure")


@pytest.mark.parametrize("hook,scene", [(2, "tiny"), (2, "medium"), (3, "tiny"), (3, "medium")])
def test_queue_wait_runs_out_and_reports_timeout(rb, orc, hook, scene):
    sc = scenes.workload_tiny()[0] if scene == "tiny" else scenes.workload_medium(level=1)[0]
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_debug_inject(rb.RT_DEBUG_SPIN_LIMIT, 20000)
    rb.rt_debug_inject(hook, 1)
    try:
        rb.rt_bvh_build(s, source=tuple(sc.tx[0]))
        with pytest.raises(rb.RtError) as ei:
            rb.rt_bvh_info(s)
        assert ei.value.code == -4  # RT_ETIMEOUT
    finally:
        rb.rt_debug_inject(hook, 0)
        rb.rt_debug_inject(rb.RT_DEBUG_SPIN_LIMIT, 0)
    # the same scene builds again, and the device is fine
    rb.rt_bvh_build(s, source=tuple(sc.tx[0]))
    assert rb.rt_bvh_info(s)["status"] == 0
    _check_usable(rb, orc)


def test_failed_allocation_reports_enomem_and_leaves_no_half_scene(rb, orc):
    sc, rays, p = scenes.workload_tiny()
    rb.rt_debug_inject(rb.RT_DEBUG_FAIL_ALLOC, 3)
    with pytest.raises(rb.RtError) as ei:
        rb.rt_scene_upload(sc.tris)
    assert ei.value.code == -2  # RT_ENOMEM
    # a scene that fails to grow is left empty: build refuses, update repairs it
    s = rb.rt_scene_upload(sc.tris[:10])
    big = scenes.workload_medium(level=1)[0]
    rb.rt_debug_inject(rb.RT_DEBUG_FAIL_ALLOC, 2)
    with pytest.raises(rb.RtError) as ei:
        rb.rt_scene_update(s, big.tris)
    assert ei.value.code == -2
    with pytest.raises(rb.RtError) as ei:
        rb.rt_bvh_build(s, source=p["source"])
    assert ei.value.code == -1  # RT_EINVAL: no buffers
    with pytest.raises(rb.RtError) as ei:
        rb.rt_trace_closest(s, torch.from_numpy(rays).cuda())
    assert ei.value.code == -3  # RT_ENOTBUILT
    rb.rt_debug_inject(rb.RT_DEBUG_FAIL_ALLOC, 0)
    rb.rt_scene_update(s, sc.tris)
    rb.rt_bvh_build(s, source=p["source"])
    assert rb.rt_bvh_info(s)["status"] == 0
    _check_usable(rb, orc)
