"""Device ray launch (Sec. III.A) and specular bounce (Sec. III.B) vs the
float64 checker (needs a GB300)."""
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


@pytest.mark.parametrize("n", [1, 7, 4096, 1_000_000])
def test_fibonacci_launch_matches_checker(rb, orc, n):
    o = (12.5, -3.0, 30.0)
    r = rb.rt_gen_rays(rb.RT_RAYS_FIBONACCI, o, n, 0.25, 750.0).cpu().numpy()
    ref = orc.fibonacci(n)[fibonacci_launch_perm(n)]      # band order: slot s holds direction perm[s]
    assert r.shape == (n, 8)
    assert np.abs(r[:, 4:7] - ref).max() < 2e-6
    assert (r[:, 0:3] == np.float32(o)).all() and (r[:, 3] == 0.25).all() and (r[:, 7] == 750.0).all()


@pytest.mark.parametrize("level", [0, 1, 2, 5, 8])
def test_icosphere_launch_matches_checker(rb, orc, level):
    n = rb.rt_ray_count(rb.RT_RAYS_ICOSPHERE, level)
    assert n == 10 * 4 ** level + 2
    r = rb.rt_gen_rays(rb.RT_RAYS_ICOSPHERE, (0, 0, 0), level).cpu().numpy()
    ref = orc.icosphere(level)[scenes.icosphere_launch_order(level)]   # tile order
    assert np.abs(r[:, 4:7] - ref).max() < 2e-6


def _bounce_chain(rb, orc, sc, rays, orders, alpha=1.0):
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, alpha=alpha, source=tuple(sc.tx[0]), max_leaf=4)
    cur = torch.from_numpy(rays).cuda()
    skip = None
    skip_np = None
    for order in range(orders + 1):
        hits = rb.rt_trace_closest(s, cur, skip=skip)
        torch.cuda.synchronize()
        h = hits.cpu().numpy()
        r_np = cur.cpu().numpy()
        ref = orc.closest_brute(sc.tris, r_np, skip=skip_np)
        compare_closest(h, ref, sc.tris, r_np, "order %d" % order)
        out_rays, out_skip, out_src, cnt = rb.rt_reflect(s, cur, hits)
        torch.cuda.synchronize()
        m = int(cnt.item())
        t, ids, _, _ = split_hits(h)
        keep = (ids >= 0) & (r_np[:, 7].astype(np.float64) - t > 0)
        assert m == keep.sum()
        src = out_src[:m].cpu().numpy()
        assert np.array_equal(src, np.nonzero(keep)[0])          # stable compaction
        nxt = out_rays[:m].cpu().numpy()
        sk = out_skip[:m].cpu().numpy()
        assert np.array_equal(sk, ids[keep])
        # the checker's float64 reflection of the GPU's hits
        refl = orc.reflect(sc.tris, r_np[keep], ids[keep], t[keep].astype(np.float64))
        scale = np.maximum(1.0, np.abs(refl[:, 0:3]).max(1, keepdims=True))
        assert np.all(np.abs(nxt[:, 0:3] - refl[:, 0:3]) <= 1e-5 * scale)
        assert np.all(np.abs(nxt[:, 4:7] - refl[:, 4:7]) <= 1e-5)
        assert np.all(np.abs(nxt[:, 7] - refl[:, 7]) <= 1e-5 * np.maximum(1.0, np.abs(refl[:, 7])))
        assert (nxt[:, 3] == 0).all()
        if m == 0:
            break
        cur = out_rays[:m].contiguous()
        skip = out_skip[:m].contiguous()
        skip_np = sk
    return s


def test_bounce_chain_tiny_city(rb, orc):
    sc, rays, _ = scenes.workload_tiny()
    _bounce_chain(rb, orc, sc, rays, orders=3)


def test_bounce_chain_medium_city_sample(rb, orc):
    sc, rays, _ = scenes.workload_medium(level=5)
    _bounce_chain(rb, orc, sc, rays, orders=3, alpha=0.7)


def test_reflect_empty_and_all_miss(rb):
    sc, rays, _ = scenes.workload_tiny()
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s)
    up = rays[rays[:, 6] > 0.5].copy()        # steep upward rays from 30 m miss everything
    cur = torch.from_numpy(up).cuda()
    hits = rb.rt_trace_closest(s, cur)
    _, _, _, cnt = rb.rt_reflect(s, cur, hits)
    torch.cuda.synchronize()
    assert int(cnt.item()) == 0
    e = torch.zeros((0, 8), dtype=torch.float32, device="cuda")
    _, _, _, cnt = rb.rt_reflect(s, e, torch.zeros((0, 4), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert int(cnt.item()) == 0
