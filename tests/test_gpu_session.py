"""Serving session: resident scenes, memory admission, continuous batching.
Every request's result must be the same alone and in the mix, and the same
as the per-call path on the same rays (needs a GB300)."""
import numpy as np
import pytest

from paper_2208_10008_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rb():
    from paper_2208_10008_gb300 import rtbvh
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    rtbvh.lib()
    return rtbvh


@pytest.fixture(scope="module")
def world(rb):
    out = []
    for seed in (1, 2, 3):
        sc = scenes.tiny_city(seed=seed)
        s = rb.rt_scene_upload(sc.tris)
        rb.rt_bvh_build(s, alpha=0.7, source=(100, 100, 25), max_leaf=4, dist_norm=1)
        out.append((sc, s))
    sc = scenes.medium_city(seed=5, n_buildings=300, size=500.0)
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, alpha=1.0, source=(250, 250, 30), max_leaf=4)
    out.append((sc, s))
    return out


def _requests(world, n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        k = int(rng.integers(0, len(world)))
        sc = world[k][0]
        x0, y0, x1, y1 = sc.area
        tx = (rng.uniform(x0, x1), rng.uniform(y0, y1), rng.uniform(10, 40))
        count = int(np.exp(rng.uniform(np.log(1000), np.log(120_000))))
        reqs.append(dict(scene=k, tx=tx, count=count, order=int(rng.integers(0, 3)), tmax=float(rng.uniform(200, 900))))
    return reqs


def test_session_same_alone_and_in_the_mix(rb, world):
    sess = rb.Session(pool_bytes=96 << 20, max_slots=3)
    ids = [sess.add_scene(s) for _, s in world]
    reqs = _requests(world, 14, seed=11)
    alone = []
    for q in reqs:
        t = sess.submit(ids[q["scene"]], q["tx"], rb.RT_RAYS_FIBONACCI, q["count"], q["order"], q["tmax"],
                        want_orders=True)
        sess.wait(t, timeout_s=60)
        h, c = sess.result(t)
        alone.append((h.copy(), c.copy(), [(oh.copy(), os_.copy()) for oh, os_ in sess.orders(t)]))
    tickets = [sess.submit(ids[q["scene"]], q["tx"], rb.RT_RAYS_FIBONACCI, q["count"], q["order"], q["tmax"],
                           want_orders=True) for q in reqs]
    for t in tickets:
        sess.wait(t, timeout_s=120)
    n_orders = 0
    for (h0, c0, o0), t in zip(alone, tickets):
        h, c = sess.result(t)
        assert np.array_equal(h.view(np.uint32), h0.view(np.uint32))
        assert np.array_equal(c, c0)
        o = sess.orders(t)
        assert len(o) == len(o0) == len(c) - 1
        for (oh, os_), (oh0, os0) in zip(o, o0):   # every reflection order, alone and in the mix
            assert np.array_equal(oh.view(np.uint32), oh0.view(np.uint32)) and np.array_equal(os_, os0)
            n_orders += 1
    assert n_orders >= 5
    st = sess.stats()
    assert st["completed"] == 2 * len(reqs) and st["failed"] == 0
    assert 1 <= st["peak_running"] <= 3 and st["p99_ms"] >= st["p50_ms"] > 0
    assert st["peak_pool_bytes"] <= st["pool_bytes"]
    # the same as the per-call path on the same launched rays, every order
    for q, (h0, c0, o0) in list(zip(reqs, alone))[:6]:
        s = world[q["scene"]][1]
        rays = rb.rt_gen_rays(rb.RT_RAYS_FIBONACCI, q["tx"], q["count"], 0.0, q["tmax"])
        hits = rb.rt_trace_closest(s, rays)
        torch.cuda.synchronize()
        assert np.array_equal(hits.cpu().numpy().view(np.uint32), h0.view(np.uint32))
        for k in range(1, q["order"] + 1):
            nr, ns, src, cnt = rb.rt_reflect(s, rays, hits)
            m = int(cnt.item())
            rays, hits = nr[:m], rb.rt_trace_closest(s, nr[:m], skip=ns[:m])
            torch.cuda.synchronize()
            oh0, os0 = o0[k - 1]
            assert m == c0[k] == len(oh0)
            assert np.array_equal(hits.cpu().numpy().view(np.uint32), oh0.view(np.uint32))
            assert np.array_equal(src[:m].cpu().numpy(), os0)
    sess.destroy()


def test_session_admission_is_bounded_by_memory(rb, world):
    n = 100_000
    need = n * (52 * 3 + 44)
    sess = rb.Session(pool_bytes=int(need * 1.5), max_slots=4)   # room for one request at a time
    sid = sess.add_scene(world[0][1])
    tickets = [sess.submit(sid, (50.0 + 10 * i, 60.0, 20.0), rb.RT_RAYS_FIBONACCI, n, 2, 500.0) for i in range(4)]
    for t in tickets:
        sess.wait(t, timeout_s=120)
    st = sess.stats()
    assert st["completed"] == 4 and st["peak_running"] == 1
    with pytest.raises(rb.RtError) as e:
        sess.submit(sid, (50.0, 60.0, 20.0), rb.RT_RAYS_FIBONACCI, 10 * n, 2, 500.0)
    assert e.value.code == -2
    with pytest.raises(rb.RtError) as e:
        sess.wait(987654, timeout_s=1)
    assert e.value.code == -1
    sess.destroy()


def test_session_release_forgets_finished_requests(rb, world):
    sess = rb.Session(pool_bytes=1 << 30, max_slots=2)   # the 2M-ray request needs about 0.4 GB
    sid = sess.add_scene(world[3][1])
    small = sess.submit(sid, (250.0, 250.0, 30.0), rb.RT_RAYS_FIBONACCI, 5000, 1, 500.0)
    sess.wait(small, timeout_s=60)
    h0, c0 = sess.result(small)
    h, c = sess.release(small)            # results stay with the caller
    assert h is h0 and np.array_equal(c, c0) and c[0] == 5000
    for call in (lambda: sess.poll(small), lambda: sess.wait(small, timeout_s=1), lambda: sess.release(small)):
        with pytest.raises(rb.RtError) as e:
            call()
        assert e.value.code == -1             # the ticket is unknown once released
    big = sess.submit(sid, (250.0, 250.0, 30.0), rb.RT_RAYS_FIBONACCI, 1 << 21, 2, 500.0, want_hits=False)
    with pytest.raises(rb.RtError) as e:     # 2M rays and two bounces cannot be done already
        sess.release(big)
    assert e.value.code == -6
    sess.wait(big, timeout_s=120)
    sess.release(big)
    st = sess.stats()
    assert st["completed"] == 2 and st["failed"] == 0 and st["p99_ms"] >= st["p50_ms"] > 0
    sess.destroy()
