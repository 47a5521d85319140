"""Range-limited builds (Sec. II.B, the ray action range) on the device (needs
a GB300): a tree over only the triangles within the range of the source
returns the same hits as the full tree and as brute force over all
triangles, for direct and reflected rays whose paths stay within the range."""
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


def _box_dist(tris, s):
    lo = tris.min(axis=1).astype(np.float64)
    hi = tris.max(axis=1).astype(np.float64)
    d = np.maximum(np.maximum(lo - s, s - hi), 0.0)
    return np.sqrt((d * d).sum(1))


@pytest.mark.parametrize("alpha", [1.0, 0.7])
def test_range_tree_hits_equal_full_tree_and_brute_force(rb, orc, alpha):
    sc = scenes.medium_city(seed=2)
    src = tuple(float(v) for v in sc.tx[0])
    R = 250.0
    full = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(full, alpha=alpha, dist_norm=1, source=src, max_leaf=4)
    part = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(part, alpha=alpha, dist_norm=1, source=src, max_leaf=4, range=R)
    info = rb.rt_bvh_info(part)
    d = _box_dist(sc.tris, np.array(src))
    assert info["n_tri"] == sc.n_tri and 0 < info["n_built"] < sc.n_tri
    assert abs(info["n_built"] - (d <= R).sum()) <= (np.abs(d - R) < 1e-2).sum()
    assert info["status"] == 0 and info["n_leaves"] == info["n_bvh2_internal"] + 1
    # the tree holds exactly the selected triangles (input ids)
    ex = rb.rt_bvh_export(part)
    prims = ex["prims"][: info["n_built"]]
    assert (ex["prims"][info["n_built"]:] == -1).all()
    assert len(np.unique(prims)) == info["n_built"] and (d[prims] <= R * 1.0001).all()
    # direct rays and two bounces, paths within R
    rays = torch.from_numpy(scenes.make_rays(src, scenes.icosphere_directions(6), 0.0, R)).cuda()
    skip = None
    for order in range(3):
        hp = rb.rt_trace_closest(part, rays, skip=skip)
        hf = rb.rt_trace_closest(full, rays, skip=skip)
        torch.cuda.synchronize()
        assert torch.equal(hp.view(torch.int32), hf.view(torch.int32)), "order %d" % order
        r_np = rays.cpu().numpy()
        if order == 0:
            ref = orc.closest_brute(sc.tris, r_np)
            compare_closest(hp.cpu().numpy(), ref, sc.tris, r_np, "range tree, direct")
        out, oskip, _, cnt = rb.rt_reflect(part, rays, hp)
        m = int(cnt.item())
        if m == 0:
            break
        rays, skip = out[:m].contiguous(), oskip[:m].contiguous()


def test_range_that_selects_nothing_gives_an_empty_tree(rb):
    sc = scenes.medium_city(seed=2)
    s = rb.rt_scene_upload(sc.tris)
    far = (50_000.0, 50_000.0, 30.0)
    rb.rt_bvh_build(s, source=far, max_leaf=4, range=100.0)
    info = rb.rt_bvh_info(s)
    assert info["n_built"] == 0 and info["status"] == 0
    rays = torch.from_numpy(scenes.make_rays(far, scenes.fibonacci_directions(1000), 0.0, 100.0)).cuda()
    h = rb.rt_trace_closest(s, rays)
    torch.cuda.synchronize()
    assert (h[:, 1].view(torch.int32) == -1).all()
    # range 0: every triangle again
    rb.rt_bvh_build(s, source=far, max_leaf=4, range=0.0)
    assert rb.rt_bvh_info(s)["n_built"] == sc.n_tri


def test_range_build_refuses_graph_capture(rb):
    sc = scenes.tiny_city(seed=1)
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, source=(100.0, 100.0, 30.0), max_leaf=4)
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(g, stream=st):  # the refusal enqueues nothing; the capture ends empty
        try:
            rb.rt_bvh_build(s, source=(100.0, 100.0, 30.0), max_leaf=4, range=50.0, stream=st)
        except rb.RtError as e:
            err = e
    assert err is not None and "captured" in str(err)
