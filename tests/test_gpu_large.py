"""The large metro at full size (about 13.2 million triangles; needs a
GB300): build with the Eq. 2 cost, check the tree's counts, check any-hit
against closest-hit on a ray sample, and compare a few hundred rays with
the float64 brute force over every triangle."""
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


def test_metro_full_size(rb, orc):
    sc = scenes.metro_city()
    assert sc.n_tri > 13_000_000
    s = rb.rt_scene_upload(sc.tris)
    centre = (10_000.0, 10_000.0, 30.0)
    rb.rt_bvh_build(s, alpha=0.7, source=centre, max_leaf=4, bins=16, dist_norm=1)
    rb.rt_bvh_build(s, alpha=0.7, source=centre, max_leaf=4, bins=16, dist_norm=1)  # timed (buffers exist)
    info = rb.rt_bvh_info(s)
    print("metro: %d triangles, build %.2f ms, depth %d, %d traversal nodes" % (
        info["n_tri"], info["build_ms"], info["depth2"], info["n_wide"]))
    assert info["status"] == 0 and info["n_tri"] == sc.n_tri
    assert info["n_leaves"] == info["n_bvh2_internal"] + 1 and info["max_leaf_size"] <= 4
    # transmitter launches in the densest area + random rays over the whole metro
    rng = np.random.default_rng(55)
    tx = np.array([sc.tris[:, :, 0].mean(), sc.tris[:, :, 1].mean(), 25.0])
    launch = scenes.make_rays(tx, scenes.fibonacci_directions(32768), 0.0, 3000.0)
    rnd = scenes.random_rays(sc, 32768, seed=56, tmax=2000.0)
    rays = np.concatenate([launch, rnd])
    r = torch.from_numpy(rays).cuda()
    h = rb.rt_trace_closest(s, r)
    o = rb.rt_trace_any(s, r)
    torch.cuda.synchronize()
    hits, occl = h.cpu().numpy(), o.cpu().numpy()
    ids = hits[:, 1].view(np.int32)
    assert np.array_equal(occl != 0, ids >= 0)  # any-hit == closest t < tmax
    assert (ids >= 0).mean() > 0.3
    sample = np.concatenate([np.arange(0, 32768, 256), 32768 + np.arange(0, 32768, 256)])
    ref = orc.closest_brute(sc.tris, rays[sample])
    compare_closest(hits[sample], ref, sc.tris, rays[sample], "metro sample")
    s.destroy()
