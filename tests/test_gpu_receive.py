"""Receiving-sphere reception (Sec. III.C, Eq. 4) on the device vs the
float64 checker (needs a GB300).  The checker takes the device's own rays and
hit distances as input (reception is a function of them), so every order is
checked on exactly what the device traced."""
import math

import numpy as np
import pytest

from paper_2208_10008_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 2e-3  # metres: float32 coordinates of a kilometre-scale scene
R0 = 500.0


@pytest.fixture(scope="module")
def rb():
    from paper_2208_10008_gb300 import rtbvh
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    rtbvh.lib()
    return rtbvh


def _receivers(sc):
    # a 32 x 32 ground grid at 1.5 m, plus a cloud around the transmitter
    rng = np.random.default_rng(11)
    near = np.asarray(sc.tx[0], np.float64) + rng.uniform(-60, 60, (256, 3)) * np.array([1, 1, 0.4])
    return np.concatenate([scenes.receiver_grid(1000.0, 32, 1.5), near.astype(np.float32)])


def _check(orc, rec, count, rays_np, hit_t, rx, delta, max_records, ray_subset=None):
    c = int(count.item())
    assert 0 <= c <= max_records
    r = rec[:c].cpu().numpy()
    pairs_gpu = [(int(a), int(b)) for a, b in r[:, :2]]
    got = set(pairs_gpu)
    assert len(got) == c, "a pair was reported twice"
    if ray_subset is not None:
        keep = np.zeros(len(rays_np), bool)
        keep[ray_subset] = True
        got = {p for p in got if keep[p[0]]}
        sub = np.asarray(ray_subset)
        pairs, vals = orc.receive(rays_np[sub], hit_t[sub], rx, delta, R0, tol=TOL)
        pairs = pairs.copy()
        pairs[:, 0] = sub[pairs[:, 0]]
    else:
        pairs, vals = orc.receive(rays_np, hit_t, rx, delta, R0, tol=TOL)
    sure = {(int(i), int(j)) for i, j, cl in pairs if cl == 1}
    near = {(int(i), int(j)): v for (i, j, _), v in zip(pairs, vals)}
    assert sure <= got, "missed %d received pairs" % len(sure - got)
    assert got <= set(near), "%d pairs the checker does not receive" % len(got - set(near))
    l = r[:, 2].copy().view(np.float32).astype(np.float64)
    dist = r[:, 3].copy().view(np.float32).astype(np.float64)
    for k, p in enumerate(pairs_gpu):
        if p in near:
            v = near[p]
            assert abs(l[k] - v[0]) <= 1e-5 * v[0] + TOL
            assert abs(dist[k] - v[1]) <= TOL
    return len(sure)


def test_receive_direct_rays_medium_city(rb, orc):
    sc, rays_np, p = scenes.workload_medium(level=6)
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, alpha=0.7, dist_norm=1, source=p["source"], max_leaf=4)
    rays = torch.from_numpy(rays_np).cuda()
    hits = rb.rt_trace_closest(s, rays)
    rx = _receivers(sc)
    delta = math.atan(2.0) / 2 ** 6
    rs = rb.rt_rxset_create(rx, R0 * delta / math.sqrt(3.0))
    rec, cnt = rb.rt_receive(rs, rays, hits, delta, R0, max_records=1 << 16)
    torch.cuda.synchronize()
    n_sure = _check(orc, rec, cnt, rays_np, hits.cpu().numpy()[:, 0], rx, delta, 1 << 16)
    assert n_sure > 100


def test_receive_after_reflection_uses_device_count(rb, orc):
    sc, rays_np, p = scenes.workload_medium(level=5)
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, alpha=0.7, dist_norm=1, source=p["source"], max_leaf=4)
    rays = torch.from_numpy(rays_np).cuda()
    hits = rb.rt_trace_closest(s, rays)
    out_rays, out_skip, _, cnt = rb.rt_reflect(s, rays, hits)
    hits1 = rb.rt_trace_closest(s, out_rays, skip=out_skip)
    rx = _receivers(sc)
    delta = math.atan(2.0) / 2 ** 5
    rs = rb.rt_rxset_create(rx, R0 * delta / math.sqrt(3.0))
    # n is the uncompacted size; the device count limits the rays taken
    rec, c = rb.rt_receive(rs, out_rays, hits1, delta, R0, n_dev=cnt, max_records=1 << 16)
    torch.cuda.synchronize()
    m = int(cnt.item())
    assert 0 < m < len(rays_np)
    r1 = out_rays[:m].cpu().numpy()
    assert (r1[:, 7] < R0).all()  # the path so far: l starts at R0 - tmax
    got_rays = rec[: int(c.item()), 0].cpu().numpy()
    assert (got_rays < m).all()
    n_sure = _check(orc, rec, c, r1, hits1[:m].cpu().numpy()[:, 0], rx, delta, 1 << 16)
    assert n_sure > 10


def test_receive_record_overflow_and_empty(rb, orc):
    sc, rays_np, p = scenes.workload_medium(level=6)
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, source=p["source"], max_leaf=4)
    rays = torch.from_numpy(rays_np).cuda()
    hits = rb.rt_trace_closest(s, rays)
    rx = _receivers(sc)
    delta = math.atan(2.0) / 2 ** 6
    rs = rb.rt_rxset_create(rx, R0 * delta / math.sqrt(3.0))
    full, cf = rb.rt_receive(rs, rays, hits, delta, R0, max_records=1 << 16)
    small, cs = rb.rt_receive(rs, rays, hits, delta, R0, max_records=7)
    torch.cuda.synchronize()
    assert int(cs.item()) == int(cf.item()) > 7
    a = {tuple(x) for x in full[: int(cf.item()), :2].cpu().numpy().tolist()}
    b = {tuple(x) for x in small[:7, :2].cpu().numpy().tolist()}
    assert len(b) == 7 and b <= a
    empty, ce = rb.rt_receive(rs, rays[:0], hits[:0], delta, R0, max_records=4)
    torch.cuda.synchronize()
    assert int(ce.item()) == 0
    with pytest.raises(rb.RtError):  # spheres larger than the set was built for
        rb.rt_receive(rs, rays, hits, 2 * delta, R0, max_records=4)


def test_receive_full_size_sampled(rb, orc):
    # the bench's configuration: icosphere level 8 (655,362 rays), 64 x 64
    # receivers at 1.5 m over the medium city; the checker runs on a sample
    sc, rays_np, p = scenes.workload_medium(level=8)
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, alpha=0.7, dist_norm=1, source=p["source"], max_leaf=4)
    rays = torch.from_numpy(rays_np).cuda()
    hits = rb.rt_trace_closest(s, rays)
    rx = scenes.receiver_grid(1000.0, 64, 1.5)
    delta = math.atan(2.0) / 2 ** 8
    rs = rb.rt_rxset_create(rx, R0 * delta / math.sqrt(3.0))
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    rec, cnt = rb.rt_receive(rs, rays, hits, delta, R0, max_records=1 << 18, stats=stats)
    torch.cuda.synchronize()
    c = int(cnt.item())
    assert c > 0
    cells, entries = stats.cpu().tolist()
    assert cells > 0 and entries >= c  # every reported pair was an entry tested
    # every ray that received something, plus a random sample of the others
    rng = np.random.default_rng(5)
    hit_rays = np.unique(rec[:c, 0].cpu().numpy())
    sample = np.union1d(hit_rays[:2000], rng.choice(len(rays_np), 6000, replace=False))
    _check(orc, rec, cnt, rays_np, hits.cpu().numpy()[:, 0], rx, delta, 1 << 18, ray_subset=sample)


def _oracle_by_delta(orc, rays_np, hit_t, rx, delta_ray):
    # the checker takes one delta per call: group the rays by their delta
    out_p, out_v = [], []
    for d in np.unique(delta_ray):
        idx = np.nonzero(delta_ray == d)[0]
        p, v = orc.receive(rays_np[idx], hit_t[idx], rx, float(d), R0, tol=TOL)
        p = p.copy()
        p[:, 0] = idx[p[:, 0]]
        out_p.append(p)
        out_v.append(v)
    return np.concatenate(out_p), np.concatenate(out_v)


def test_batch_reception_every_order_matches_checker(rb, orc):
    # four transmitters with different Fibonacci counts (so different delta:
    # sqrt(4 pi / N)) and two reflection orders; each ray keeps its
    # transmitter's delta through the bounces
    sc = scenes.medium_city(seed=2)
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, source=(500.0, 500.0, 20.0), max_leaf=4)
    tx = np.array([[500, 500, 30], [300, 620, 12], [700, 380, 25], [450, 260, 18]], np.float32)
    counts = np.array([20000, 8000, 30000, 12000], np.int64)
    rx = scenes.receiver_grid(1000.0, 24, 1.5)
    b = rb.Batch(s, tx, counts, kind=rb.RT_RAYS_FIBONACCI, max_order=2, tmax=R0, rx_pos=rx, receive=True,
                 max_rx_records=1 << 16)
    for _ in range(3):  # direct run, graph capture, graph replay
        b.run()
    torch.cuda.synchronize()
    st = b.stats()
    dtx = np.sqrt(4 * np.pi / counts.astype(np.float64)).astype(np.float32)
    d_prev = np.repeat(dtx, counts)
    total = 0
    for k in range(3):
        rays, hits, src, n = b.order(k)
        rays_np = rays.cpu().numpy()
        hit_t = hits.cpu().numpy()[:, 0]
        d_ray = d_prev if k == 0 else d_prev[src.cpu().numpy()]
        rec, c = b.received(k)
        assert c == st["received"][k] and c <= 1 << 16
        r = rec.cpu().numpy()
        got = {(int(a), int(bb)) for a, bb in r[:, :2]}
        assert len(got) == c
        pairs, vals = _oracle_by_delta(orc, rays_np, hit_t, rx, d_ray)
        sure = {(int(i), int(j)) for i, j, cl in pairs if cl == 1}
        near = {(int(i), int(j)) for i, j, _ in pairs}
        assert sure <= got, "order %d: missed %d" % (k, len(sure - got))
        assert got <= near, "order %d: %d extra" % (k, len(got - near))
        total += c
        d_prev = d_ray
    assert total > 50
