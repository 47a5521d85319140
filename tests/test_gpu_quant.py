"""64-byte quantised traversal nodes (needs a GB300): the walk over them
returns exactly the hits of the 128-byte float-node walk (their decoded
boxes contain the exact ones, and the hit rule does not depend on the tree)
and of brute force."""
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


def _same(a, b):
    return torch.equal(a.contiguous().view(torch.int32), b.contiguous().view(torch.int32))


@pytest.mark.parametrize("alpha,offset", [(0.7, 0.0), (1.0, 0.0), (1.0, 1.0e5)])
def test_quantised_walk_equals_float_walk(rb, orc, alpha, offset):
    sc = scenes.medium_city(seed=2)
    tris = sc.tris + np.float32(offset) * np.array([1, 1, 0], np.float32)  # far from the origin too
    src = np.array(sc.tx[0]) + offset * np.array([1, 1, 0])
    s = rb.rt_scene_upload(tris)
    rb.rt_bvh_build(s, alpha=alpha, dist_norm=1, source=tuple(src), max_leaf=4, quantize=1)
    assert rb.rt_bvh_info(s)["status"] == 0
    rays_np = np.concatenate([scenes.make_rays(src, scenes.icosphere_directions(6), 0.0, 500.0),
                              scenes.random_rays(sc, 20000, seed=9, tmax=800.0)])
    rays_np[:, 0:2] += np.float32(offset) * (np.arange(len(rays_np)) >= 40962)[:, None]
    rays = torch.from_numpy(rays_np).cuda()
    hf = rb.rt_trace_closest(s, rays)
    hq = rb.rt_trace_closest(s, rays, flags=rb.RT_QUANTIZED_NODES)
    of = rb.rt_trace_any(s, rays)
    oq = rb.rt_trace_any(s, rays, flags=rb.RT_QUANTIZED_NODES)
    torch.cuda.synchronize()
    assert _same(hf, hq)
    assert torch.equal(of, oq)
    sample = np.arange(0, len(rays_np), 97)
    ref = orc.closest_brute(tris, rays_np[sample])
    compare_closest(hq.cpu().numpy()[sample], ref, tris, rays_np[sample], "quantised walk")
    # the decoded boxes are never smaller: the walk cannot test fewer triangles in total
    sf = torch.zeros((len(rays_np), 2), dtype=torch.int32, device="cuda")
    sq = torch.zeros_like(sf)
    rb.rt_trace_closest(s, rays, stats=sf)
    rb.rt_trace_closest(s, rays, stats=sq, flags=rb.RT_QUANTIZED_NODES)
    torch.cuda.synchronize()
    assert sq[:, 0].sum().item() > 0 and sq.double().mean(0)[1] >= 0.95 * sf.double().mean(0)[1]


def test_quantised_walk_flat_and_tiny_scenes(rb, orc):
    # the tiny city: boxes and a flat ground (zero extent on z for its node)
    sc, rays_np, p = scenes.workload_tiny()
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, source=p["source"], max_leaf=2, quantize=1)
    rays = torch.from_numpy(rays_np).cuda()
    hq = rb.rt_trace_closest(s, rays, flags=rb.RT_QUANTIZED_NODES)
    torch.cuda.synchronize()
    compare_closest(hq.cpu().numpy(), orc.closest_brute(sc.tris, rays_np), sc.tris, rays_np, "quantised tiny")
    # ground only: every node box is flat in z
    g = np.array([[[0, 0, 0], [100, 0, 0], [0, 100, 0]], [[100, 0, 0], [100, 100, 0], [0, 100, 0]]], np.float32)
    s2 = rb.rt_scene_upload(g)
    rb.rt_bvh_build(s2, max_leaf=1, quantize=1)
    down = scenes.make_rays((30.0, 40.0, 10.0), scenes.fibonacci_directions(2000), 0.0, 100.0)
    r2 = torch.from_numpy(down).cuda()
    h2 = rb.rt_trace_closest(s2, r2, flags=rb.RT_QUANTIZED_NODES)
    torch.cuda.synchronize()
    compare_closest(h2.cpu().numpy(), orc.closest_brute(g, down), g, down, "quantised ground")


def test_quantised_flag_needs_a_quantised_build(rb):
    sc, rays_np, p = scenes.workload_tiny()
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, source=p["source"], max_leaf=2)
    rays = torch.from_numpy(rays_np).cuda()
    with pytest.raises(rb.RtError):
        rb.rt_trace_closest(s, rays, flags=rb.RT_QUANTIZED_NODES)
    rb.rt_bvh_build(s, source=p["source"], max_leaf=2, quantize=1)
    rb.rt_trace_closest(s, rays, flags=rb.RT_QUANTIZED_NODES)
    rb.rt_bvh_build(s, source=p["source"], max_leaf=2)  # a later build without: refused again
    with pytest.raises(rb.RtError):
        rb.rt_trace_closest(s, rays, flags=rb.RT_QUANTIZED_NODES)
    torch.cuda.synchronize()


def test_quantised_nodes_of_a_range_tree(rb):
    # both options together: a tree pruned to the range of its source, with
    # its 64-byte nodes; direct rays within the range hit exactly as on the
    # whole-scene float tree
    sc = scenes.medium_city(seed=2)
    src = tuple(float(v) for v in sc.tx[0])
    full = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(full, alpha=0.7, dist_norm=1, source=src, max_leaf=4)
    part = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(part, alpha=0.7, dist_norm=1, source=src, max_leaf=4, range=300.0, quantize=1)
    assert 0 < rb.rt_bvh_info(part)["n_built"] < sc.n_tri
    rays = torch.from_numpy(scenes.make_rays(src, scenes.icosphere_directions(6), 0.0, 300.0)).cuda()
    hf = rb.rt_trace_closest(full, rays)
    hq = rb.rt_trace_closest(part, rays, flags=rb.RT_QUANTIZED_NODES)
    torch.cuda.synchronize()
    assert _same(hf, hq)
