"""GPU path vs the float64 checker, through the C ABI (needs a GB300)."""
import numpy as np
import pytest

from paper_2208_10008_gb300 import scenes
from helpers import compare_closest, split_hits

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


def trace(rb, scene, rays, **kw):
    h = rb.rt_trace_closest(scene, dev(rays), **kw)
    torch.cuda.synchronize()
    return h.cpu().numpy()


def build(rb, tris, **kw):
    s = rb.rt_scene_upload(tris)
    rb.rt_bvh_build(s, **kw)
    info = rb.rt_bvh_info(s)
    assert info["status"] == 0
    return s, info


# ------------------------------------------------------------------ C1 tiny city
@pytest.mark.parametrize("max_leaf", [1, 4, 8, 15])
def test_tiny_city_all_rays_vs_brute(rb, orc, max_leaf):
    sc, rays, p = scenes.workload_tiny()
    s, info = build(rb, sc.tris, alpha=1.0, source=p["source"], max_leaf=max_leaf)
    assert info["max_leaf_size"] <= max_leaf
    ref = orc.closest_brute(sc.tris, rays)
    nf = torch.zeros(1, dtype=torch.int32, device="cuda")
    h = trace(rb, s, rays, n_flagged=nf)
    n, nh, nt = compare_closest(h, ref, sc.tris, rays, "tiny")
    assert nh > 1000
    print("tiny max_leaf=%d flagged=%d ties=%d" % (max_leaf, int(nf.item()), nt))


def test_tiny_city_any_hit(rb, orc):
    sc, rays, p = scenes.workload_tiny()
    rays = rays.copy()
    rays[:, 7] = np.random.default_rng(3).uniform(1, 150, len(rays)).astype(np.float32)
    s, _ = build(rb, sc.tris, alpha=1.0, source=p["source"])
    occ = rb.rt_trace_any(s, dev(rays))
    torch.cuda.synchronize()
    ref = orc.any_brute(sc.tris, rays)
    assert (occ.cpu().numpy() == ref).all()
    h = trace(rb, s, rays)
    assert ((split_hits(h)[1] >= 0) == (occ.cpu().numpy() == 1)).all()


# ------------------------------------------------------------------ C2 medium city
@pytest.mark.parametrize("alpha,dist_norm", [(1.0, 0), (0.7, 1), (0.4, 1), (0.4, 0), (0.0, 0)])
def test_medium_city_full_icosphere(rb, orc, alpha, dist_norm):
    sc, rays, p = scenes.workload_medium()
    s, info = build(rb, sc.tris, alpha=alpha, source=p["source"], max_leaf=4, bins=16, dist_norm=dist_norm)
    # the checker's BVH walk equals its brute force (pinned); use it at full size
    ob = orc.Bvh(sc.tris, alpha=1.0, max_leaf=4)
    ref = ob.closest(rays)
    nf = torch.zeros(1, dtype=torch.int32, device="cuda")
    h = trace(rb, s, rays, n_flagged=nf)
    n, nh, nt = compare_closest(h, ref, sc.tris, rays, "medium a=%g dn=%d" % (alpha, dist_norm))
    print("medium a=%g dn=%d: rays %d hits %d ties %d flagged %d info %s" % (
        alpha, dist_norm, n, nh, nt, int(nf.item()), info))
    # brute force on a sample as well
    k = np.random.default_rng(0).choice(len(rays), 3000, replace=False)
    bref = orc.closest_brute(sc.tris, rays[k])
    compare_closest(h[k], bref, sc.tris, rays[k], "medium brute")


def test_medium_city_random_rays_and_any(rb, orc):
    sc, _, p = scenes.workload_medium(level=2)
    rays = scenes.random_rays(sc, 200_000, seed=21, tmax=300.0)
    rays[::7, 7] = np.inf
    s, _ = build(rb, sc.tris, alpha=0.7, source=p["source"], dist_norm=1)
    ob = orc.Bvh(sc.tris, alpha=1.0, max_leaf=4)
    ref = ob.closest(rays)
    compare_closest(trace(rb, s, rays), ref, sc.tris, rays, "random")
    occ = rb.rt_trace_any(s, dev(rays))
    torch.cuda.synchronize()
    assert (occ.cpu().numpy() == (ref.id >= 0)).all()


# ------------------------------------------------------------------ tree structure
def _tree_checks(ex, tris, max_leaf):
    prims = ex["prims"]
    assert sorted(prims.tolist()) == list(range(len(tris)))
    lc = ex["leaf_count"]
    assert (lc >= 1).all() and (lc <= max_leaf).all() and lc.sum() == len(tris)
    child = ex["child"]
    boxes = ex["boxes"]
    tb = tris.astype(np.float32)

    def gather(c):
        out = []
        st = [c]
        while st:
            x = st.pop()
            if x < 0:
                l = -1 - x
                out.extend(prims[ex["leaf_first"][l]: ex["leaf_first"][l] + lc[l]])
            else:
                st.extend(child[x])
        return out

    # every child box is exactly the AABB of its triangles (hence inside its parent)
    rng = np.random.default_rng(0)
    sample = rng.choice(len(child), min(len(child), 400), replace=False) if len(child) else []
    for i in sample:
        for s in range(2):
            ids = gather(child[i][s])
            pts = tb[ids].reshape(-1, 3)
            assert np.array_equal(boxes[i][6 * s: 6 * s + 3], pts.min(0)), i
            assert np.array_equal(boxes[i][6 * s + 3: 6 * s + 6], pts.max(0)), i


@pytest.mark.parametrize("alpha,dist_norm,max_leaf", [(1.0, 0, 4), (0.7, 1, 4), (0.4, 0, 2), (1.0, 0, 1)])
def test_bvh_structure_and_quality(rb, orc, alpha, dist_norm, max_leaf):
    sc, _, p = scenes.workload_medium(level=1)
    s, info = build(rb, sc.tris, alpha=alpha, source=p["source"], max_leaf=max_leaf, bins=32,
                    dist_norm=dist_norm)
    ex = rb.rt_bvh_export(s)
    _tree_checks(ex, sc.tris, max_leaf)
    src = p["source"]
    c_gpu = orc.tree_cost(sc.tris, ex["child"], ex["leaf_first"], ex["leaf_count"], ex["prims"], alpha,
                          src, dist_norm=dist_norm)
    ob = orc.Bvh(sc.tris, alpha=alpha, source=src, max_leaf=max_leaf, dist_norm=dist_norm)
    c_ref = ob.cost()
    print("quality a=%g dn=%d leaf=%d: gpu %.6g exact-sweep %.6g ratio %.4f depth %d/%d" % (
        alpha, dist_norm, max_leaf, c_gpu, c_ref, c_gpu / c_ref, info["depth2"], ob.info()["depth"]))
    assert c_gpu <= 1.10 * c_ref  # reading c6, at every alpha


def test_build_deterministic(rb):
    sc, _, p = scenes.workload_medium(level=1)
    s1, _ = build(rb, sc.tris, alpha=0.7, source=p["source"], dist_norm=1)
    s2, _ = build(rb, sc.tris, alpha=0.7, source=p["source"], dist_norm=1)
    e1, e2 = rb.rt_bvh_export(s1), rb.rt_bvh_export(s2)
    for k in ("child", "leaf_first", "leaf_count", "prims", "boxes"):
        assert np.array_equal(e1[k], e2[k]), k


# ------------------------------------------------------------------ edge cases
def test_empty_inputs(rb, orc):
    sc, rays, p = scenes.workload_tiny()
    s, _ = build(rb, sc.tris)
    h = rb.rt_trace_closest(s, dev(rays[:0]))
    torch.cuda.synchronize()
    assert h.shape == (0, 4)
    empty = rb.rt_scene_upload(np.zeros((0, 3, 3), np.float32))
    rb.rt_bvh_build(empty)
    h = trace(rb, empty, rays)
    t, ids, _, _ = split_hits(h)
    assert (ids == -1).all() and np.isinf(t).all()


@pytest.mark.parametrize("n_tri", [1, 2, 3, 5, 16, 17])
def test_tiny_scenes_root_leaf(rb, orc, n_tri):
    sc, rays, p = scenes.workload_tiny()
    tris = sc.tris[-n_tri:].copy()     # includes the ground
    s, info = build(rb, tris, max_leaf=4)
    compare_closest(trace(rb, s, rays), orc.closest_brute(tris, rays), tris, rays, "n_tri=%d" % n_tri)


@pytest.mark.parametrize("n", [1, 31, 127, 129, 1000, 4097])
def test_ragged_ray_counts(rb, orc, n):
    sc, rays, p = scenes.workload_tiny()
    rng = np.random.default_rng(n)
    r = scenes.random_rays(sc, n, seed=n, tmax=500.0)
    s, _ = build(rb, sc.tris, alpha=1.0)
    compare_closest(trace(rb, s, r), orc.closest_brute(sc.tris, r), sc.tris, r, "n=%d" % n)


def test_invalid_rays_miss(rb):
    sc, rays, p = scenes.workload_tiny()
    r = rays[:6].copy()
    r[0, 0] = np.nan
    r[1, 4] = np.inf
    r[2, 3], r[2, 7] = 5.0, 5.0
    r[3, 3], r[3, 7] = 9.0, 1.0
    r[4, 4:7] = 0.0
    r[5, 7] = np.nan
    s, _ = build(rb, sc.tris)
    t, ids, _, _ = split_hits(trace(rb, s, r))
    assert (ids == -1).all() and np.isinf(t).all()
    occ = rb.rt_trace_any(s, dev(r))
    torch.cuda.synchronize()
    assert (occ.cpu().numpy() == 0).all()


def test_grazing_vertex_edge_suite(rb, orc):
    """Rays aimed exactly at vertices and edge midpoints (ties, edge grazes)."""
    sc = scenes.tiny_city(seed=1)
    v = sc.tris.reshape(-1, 3).astype(np.float64)
    rng = np.random.default_rng(6)
    pick = rng.choice(len(v), 3000)
    tgt = np.concatenate([v[pick], 0.5 * (v[pick] + v[rng.choice(len(v), 3000)])])
    o = np.array([100.0, 100.0, 30.0])
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = scenes.make_rays(o, d, 0.0, 1e4)
    s, _ = build(rb, sc.tris, alpha=1.0, max_leaf=2)
    nf = torch.zeros(1, dtype=torch.int32, device="cuda")
    h = trace(rb, s, rays, n_flagged=nf)
    compare_closest(h, orc.closest_brute(sc.tris, rays), sc.tris, rays, "grazing")
    print("grazing flagged", int(nf.item()), "of", len(rays))


def test_axis_parallel_rays(rb, orc):
    sc = scenes.tiny_city(seed=1)
    rng = np.random.default_rng(9)
    n = 6000
    o = np.stack([rng.uniform(0, 200, n), rng.uniform(0, 200, n), rng.uniform(0, 45, n)], 1)
    # snap some origins onto exact box planes so that 0 * inf appears in the slab test
    vx = sc.tris.reshape(-1, 3)
    snap = rng.choice(len(vx), n // 3)
    o[: n // 3, 0] = vx[snap, 0]
    o[n // 3: 2 * n // 3, 2] = vx[snap, 2]
    axes = np.eye(3)[rng.integers(0, 3, n)] * rng.choice([-1.0, 1.0], (n, 1))
    rays = scenes.make_rays((0, 0, 0), axes, 0.0, 1e3)
    rays[:, 0:3] = o.astype(np.float32)
    s, _ = build(rb, sc.tris, alpha=1.0)
    compare_closest(trace(rb, s, rays), orc.closest_brute(sc.tris, rays), sc.tris, rays, "axis")


def test_duplicate_and_degenerate_triangles(rb, orc):
    sc, rays, p = scenes.workload_tiny()
    tris = np.concatenate([sc.tris, sc.tris[:50], np.repeat(sc.tris[:5, :1], 3, axis=1)])
    s, _ = build(rb, tris, alpha=1.0)
    compare_closest(trace(rb, s, rays), orc.closest_brute(tris, rays), tris, rays, "dups")


def test_skip_triangle(rb, orc):
    sc, rays, p = scenes.workload_tiny()
    s, _ = build(rb, sc.tris, alpha=1.0)
    ref0 = orc.closest_brute(sc.tris, rays)
    skip = ref0.id.astype(np.int32)
    ref = orc.closest_brute(sc.tris, rays, skip=skip)
    h = trace(rb, s, rays, skip=dev(skip))
    compare_closest(h, ref, sc.tris, rays, "skip")


def test_tmax_culling_never_drops_hits_in_range(rb, orc):
    sc, rays, p = scenes.workload_tiny()
    s, _ = build(rb, sc.tris, alpha=1.0)
    full = split_hits(trace(rb, s, rays))
    for frac in (0.3, 0.7, 1.0001):
        r = rays.copy()
        fin = np.isfinite(full[0])
        r[fin, 7] = (full[0][fin] * frac).astype(np.float32)
        t, ids, _, _ = split_hits(trace(rb, s, r))
        keep = fin & (full[0] < r[:, 7])
        assert (ids[keep] == full[1][keep]).all()
        drop = fin & (full[0] >= r[:, 7])
        assert (t[drop] < r[drop, 7]).all() or (ids[drop] == -1).all()


def test_host_buffer_path_matches_device(rb):
    sc, rays, p = scenes.workload_medium(level=6)
    s, _ = build(rb, sc.tris, alpha=0.7, source=p["source"], dist_norm=1)
    hd = trace(rb, s, rays)
    pinned = torch.from_numpy(rays).pin_memory()
    hh = rb.rt_trace_closest_host(s, pinned)
    assert np.array_equal(hh.numpy().view(np.uint32), hd.view(np.uint32))
    for tile in (64, 256):  # the requested ray tile reaches the chunked walk
        hh = rb.rt_trace_closest_host(s, pinned, block=tile)
        assert np.array_equal(hh.numpy().view(np.uint32), hd.view(np.uint32))
    # page-locked hits 4 bytes off a 16-byte boundary: the walk cannot store
    # records there, so they go through the staging buffers; same bits
    n = len(rays)
    spare = torch.empty(4 * n + 1, dtype=torch.float32).pin_memory()
    odd = spare[1:].view(n, 4)
    assert odd.data_ptr() % 16 == 4
    rb.rt_trace_closest_host(s, pinned, odd)
    assert np.array_equal(odd.numpy().view(np.uint32), hd.view(np.uint32))


def test_host_buffer_path_many_chunks(rb):
    # more rays than the pipeline's two staging buffers hold at once (2 x 2^20):
    # chunks of 2^20 take the buffers in turn; every hit equals the device
    # path's, bit for bit
    sc, _, p = scenes.workload_medium(level=1)
    s, _ = build(rb, sc.tris, alpha=0.7, source=p["source"], dist_norm=1)
    rays = scenes.random_rays(sc, 4 * (1 << 20) + 12345, seed=91, tmax=300.0)
    hd = trace(rb, s, rays)
    pinned = torch.from_numpy(rays).pin_memory()
    hh = rb.rt_trace_closest_host(s, pinned, stack=32)
    assert np.array_equal(hh.numpy().view(np.uint32), hd.view(np.uint32))
    hn = rb.rt_trace_closest_host(s, rays[:777])  # pageable numpy buffers, a short batch
    assert np.array_equal(hn.view(np.uint32), hd[:777].view(np.uint32))


def test_stats_and_no_retest_flag(rb, orc):
    sc, rays, p = scenes.workload_tiny()
    s, _ = build(rb, sc.tris, alpha=1.0)
    stats = torch.zeros((len(rays), 2), dtype=torch.int32, device="cuda")
    h1 = trace(rb, s, rays, stats=stats)
    st = stats.cpu().numpy()
    assert (st[:, 0] >= 1).all() and st[:, 1].sum() > 0
    h2 = trace(rb, s, rays)
    assert np.array_equal(h1.view(np.uint32), h2.view(np.uint32))


def test_errors(rb):
    sc, rays, p = scenes.workload_tiny()
    s = rb.rt_scene_upload(sc.tris)
    with pytest.raises(rb.RtError) as e:
        rb.rt_trace_closest(s, dev(rays))
    assert e.value.code == -3
    with pytest.raises(rb.RtError) as e:
        rb.rt_bvh_build(s, alpha=1.5)
    assert e.value.code == -1
    with pytest.raises(rb.RtError):
        rb.rt_bvh_build(s, max_leaf=16)
    with pytest.raises(rb.RtError):
        rb.rt_bvh_build(s, bins=2)


def test_binding_rejects_short_output_buffers(rb):
    """A caller's output buffer smaller than the call writes is refused before
    the library is called (the kernels would write past its end)."""
    sc, rays, p = scenes.workload_tiny()
    s, _ = build(rb, sc.tris, alpha=1.0)
    r = dev(rays)
    n = r.shape[0]
    f32, i32 = dict(dtype=torch.float32, device="cuda"), dict(dtype=torch.int32, device="cuda")
    short = [
        lambda: rb.rt_trace_closest(s, r, torch.empty((n - 1, 4), **f32)),
        lambda: rb.rt_trace_closest(s, r, n_flagged=torch.empty(0, **i32)),
        lambda: rb.rt_trace_any(s, r, torch.empty(n - 1, dtype=torch.uint8, device="cuda")),
        lambda: rb.rt_trace_closest_noalloc(s, r[:16], torch.empty((15, 4), **f32)),
        lambda: rb.rt_reflect(s, r, torch.empty((n - 1, 4), **f32)),
        lambda: rb.rt_reflect(s, r, torch.empty((n, 4), **f32), out_rays=torch.empty((n - 1, 8), **f32)),
        lambda: rb.rt_reflect(s, r, torch.empty((n, 4), **f32), out_count=torch.empty(0, **i32)),
    ]
    for call in short:
        with pytest.raises(TypeError):
            call()
    rs = rb.rt_rxset_create(np.array([[100.0, 100.0, 2.0]]), 1.0)
    with pytest.raises(TypeError):
        rb.rt_receive(rs, r, torch.empty((n - 1, 4), **f32), 0.01, 100.0)
    rs.destroy()
    s.destroy()
