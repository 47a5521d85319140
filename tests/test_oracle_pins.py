"""Pins for the float64 CPU checker (oracle/) -- no GPU.

Each test ties the checker to something other than itself: a closed form, a
hand-worked example, brute force written another way, an invariant the paper
states (Sec. IV.B: the accelerated tracer finds the same paths), or a special
case that reduces to a textbook definition.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2208_10008_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def ray(o, d, tmin=0.0, tmax=np.inf):
    return np.array([*o, tmin, *d, tmax], dtype=np.float32)


TRI = np.array([[0, 0, 5], [4, 0, 5], [0, 4, 5]], dtype=np.float32)


# --------------------------------------------------------------- triangle test
def test_tri_axis_ray_closed_form(orc):
    # plane z = 5 hit straight on: t = 5, barycentrics u = x/4 (weight of v1), v = y/4 (v2)
    hit, t, u, v = orc.tri_hit(TRI, ray((1, 1, 0), (0, 0, 1)))
    assert hit and t == 5.0 and u == 0.25 and v == 0.25


def test_tri_oblique_ray_closed_form(orc):
    rng = np.random.default_rng(0)
    for _ in range(200):
        px, py = rng.uniform(0.05, 1.9, 2)
        o = np.array([rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(-4, 1)])
        p = np.array([px, py, 5.0])
        d = p - o
        d /= np.linalg.norm(d)
        r = ray(o, d)
        rd = r[4:7].astype(np.float64)
        ro = r[0:3].astype(np.float64)
        # exact plane intersection of the float32 ray: distance / cos(theta)
        t_ref = (5.0 - ro[2]) / rd[2]
        q = ro + t_ref * rd
        hit, t, u, v = orc.tri_hit(TRI, r)
        assert hit
        assert abs(t - t_ref) <= 1e-12 * t_ref
        assert abs(u - q[0] / 4) < 1e-12 and abs(v - q[1] / 4) < 1e-12


def test_tri_outside_misses(orc):
    for p in [(-0.1, 1, 5), (1, -0.1, 5), (2.1, 2.1, 5), (5, 5, 5)]:
        hit, *_ = orc.tri_hit(TRI, ray((p[0], p[1], 0), (0, 0, 1)))
        assert not hit


def test_tri_edges_and_vertices_inclusive(orc):
    for p in [(0, 0), (4, 0), (0, 4), (2, 0), (0, 2), (2, 2), (1, 3)]:
        hit, t, u, v = orc.tri_hit(TRI, ray((p[0], p[1], 0), (0, 0, 1)))
        assert hit and t == 5.0, p


def test_tri_two_sided(orc):
    h1 = orc.tri_hit(TRI, ray((1, 1, 0), (0, 0, 1)))
    h2 = orc.tri_hit(TRI, ray((1, 1, 10), (0, 0, -1)))
    assert h1[0] and h2[0] and h1[1] == h2[1] == 5.0


def test_tri_parallel_and_degenerate_miss(orc):
    assert not orc.tri_hit(TRI, ray((1, 1, 5), (1, 0, 0)))[0]      # in plane
    assert not orc.tri_hit(TRI, ray((1, 1, 3), (0, 1, 0)))[0]      # parallel
    line = np.array([[0, 0, 5], [1, 1, 5], [2, 2, 5]], np.float32)  # collinear
    assert not orc.tri_hit(line, ray((1, 1, 0), (0, 0, 1)))[0]
    point = np.array([[1, 1, 5]] * 3, np.float32)
    assert not orc.tri_hit(point, ray((1, 1, 0), (0, 0, 1)))[0]
    assert not orc.tri_hit(TRI, ray((1, 1, 0), (0, 0, 0)))[0]       # zero direction


def test_tri_parallel_threshold_scale(orc):
    """The parallel rule |det| <= 1e-14 |e1||e2||d| on both sides of the
    threshold.  For a triangle in z = 0 with e1 = (4,0,0), e2 = (0,4,0) and
    a ray (1, 0, -eps) from height h, det = 16 eps, so the ratio is eps:
    eps = 1e-8 is a real (grazing) hit at t = h / eps with u = v = 0.25;
    eps = 1e-15 counts as parallel."""
    tri0 = np.array([[0, 0, 0], [4, 0, 0], [0, 4, 0]], dtype=np.float32)
    r = ray((-1.0, 1.0, 2e-8), (1.0, 0.0, -1e-8))
    hit, t, u, v = orc.tri_hit(tri0, r)
    t_ref = float(r[2]) / -float(r[6])          # plane z = 0 from the float32 ray
    assert hit and abs(t - t_ref) <= 1e-9 * t_ref
    assert abs(u - (-1.0 + t_ref) / 4) < 1e-9 and abs(v - 0.25) < 1e-9
    assert not orc.tri_hit(tri0, ray((-1.0, 1.0, 2e-15), (1.0, 0.0, -1e-15)))[0]


# --------------------------------------------------------------- brute force
def _solve_brute(tris, rays):
    """Closest hit by solving o + t d = v0 + u e1 + v e2 with numpy.linalg.solve."""
    T = tris.astype(np.float64)
    out_t = np.full(len(rays), np.inf)
    out_id = np.full(len(rays), -1)
    margin = np.zeros(len(rays))        # how close any decision came to a boundary
    for r, ry in enumerate(rays.astype(np.float64)):
        o, d, tmin, tmax = ry[0:3], ry[4:7], ry[3], ry[7]
        best, bid, marg = np.inf, -1, np.inf
        ts = []
        for i, (v0, v1, v2) in enumerate(T):
            M = np.stack([-d, v1 - v0, v2 - v0], axis=1)
            if abs(np.linalg.det(M)) < 1e-9:
                continue
            t, u, v = np.linalg.solve(M, o - v0)
            marg = min(marg, abs(u), abs(v), abs(1 - u - v), abs(t - tmin), abs(t - tmax))
            if u >= 0 and v >= 0 and u + v <= 1 and tmin < t < tmax:
                ts.append(t)
                if t < best:
                    best, bid = t, i
        ts.sort()
        if len(ts) > 1:
            marg = min(marg, (ts[1] - ts[0]) / max(ts[0], 1e-300))
        out_t[r], out_id[r], margin[r] = best, bid, marg
    return out_t, out_id, margin


def test_brute_matches_linear_solve(orc):
    rng = np.random.default_rng(1)
    tris = rng.uniform(-10, 10, size=(40, 3, 3)).astype(np.float32)
    o = rng.uniform(-12, 12, size=(400, 3))
    d = rng.normal(size=(400, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([o, np.zeros((400, 1)), d, np.full((400, 1), 30.0)], axis=1).astype(np.float32)
    h = orc.closest_brute(tris, rays)
    t_ref, id_ref, marg = _solve_brute(tris, rays)
    ok = marg > 1e-9
    assert ok.mean() > 0.95
    assert (h.id[ok] == id_ref[ok]).all()
    hit = ok & (id_ref >= 0)
    assert hit.sum() > 50
    assert np.allclose(h.t[hit], t_ref[hit], rtol=1e-11, atol=0)


def test_ground_only_city_closed_form(orc):
    A = 1000.0
    tris = np.asarray(scenes._ground(0, 0, A, A), np.float32)
    rng = np.random.default_rng(2)
    n = 3000
    o = np.stack([rng.uniform(-200, 1200, n), rng.uniform(-200, 1200, n), rng.uniform(1, 50, n)], 1)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = scenes.make_rays((0, 0, 0), d, 0.0, np.inf)
    rays[:, 0:3] = o.astype(np.float32)
    h = orc.closest_brute(tris, rays)
    r64 = rays.astype(np.float64)
    tz = -r64[:, 2] / r64[:, 6]
    land = r64[:, 0:3] + tz[:, None] * r64[:, 4:7]
    inside = (r64[:, 6] < 0) & (land[:, 0] >= 0) & (land[:, 0] <= A) & (land[:, 1] >= 0) & (land[:, 1] <= A)
    edge = (np.abs(land[:, 0]) < 1e-6) | (np.abs(land[:, 0] - A) < 1e-6) | (np.abs(land[:, 1]) < 1e-6) | (np.abs(land[:, 1] - A) < 1e-6)
    ok = ~edge
    assert ((h.id >= 0)[ok] == inside[ok]).all()
    sel = ok & inside
    assert np.allclose(h.t[sel], tz[sel], rtol=1e-12, atol=0)


def _slab_entry(o, d, lo, hi):
    t0, t1 = -np.inf, np.inf
    for a in range(3):
        if d[a] == 0:
            if o[a] < lo[a] or o[a] > hi[a]:
                return np.inf, np.inf
            continue
        ta, tb = (lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return t0, t1


def test_single_box_slab_entry(orc):
    lo, hi = np.array([10.0, 20.0, 0.0]), np.array([25.0, 32.0, 17.0])
    tris = np.asarray(scenes._box(lo[0], lo[1], hi[0], hi[1], hi[2]), np.float32)
    rng = np.random.default_rng(3)
    n = 3000
    o = rng.uniform(-30, 70, size=(n, 3))
    o[:, 2] = rng.uniform(-10, 40, n)
    aim = rng.uniform(lo - 3, hi + 3)
    d = aim - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([o, np.zeros((n, 1)), d, np.full((n, 1), np.inf)], 1).astype(np.float32)
    h = orc.closest_brute(tris, rays)
    checked = 0
    for r in range(n):
        ro, rd = rays[r, 0:3].astype(np.float64), rays[r, 4:7].astype(np.float64)
        if np.all(ro >= lo) and np.all(ro <= hi):
            continue  # origin inside the box
        t0, t1 = _slab_entry(ro, rd, lo, hi)
        p = ro + t0 * rd
        # distance of the entry point to the nearest box edge (grazing rays are skipped)
        on = np.sort(np.minimum(np.abs(p - lo), np.abs(p - hi)))
        if np.isfinite(t0) and t0 <= t1 and on[1] < 1e-6:
            continue
        if np.isfinite(t0) and t0 < t1 and t0 > 0:
            assert h.id[r] >= 0 and abs(h.t[r] - t0) <= 1e-10 * t0, r
            checked += 1
        else:
            assert h.id[r] < 0, r
    assert checked > 500


def test_shared_edge_tie_lowest_id(orc):
    # unit square in z = 2 split along its diagonal; the diagonal is shared
    sq = np.array([[[0, 0, 2], [1, 0, 2], [1, 1, 2]], [[0, 0, 2], [1, 1, 2], [0, 1, 2]]], np.float32)
    for p in [(0.5, 0.5), (0.25, 0.25), (0.0, 0.0), (1.0, 1.0)]:
        for order in (sq, sq[::-1].copy()):
            h = orc.closest_brute(order, ray((p[0], p[1], 0), (0, 0, 1))[None])
            assert h.id[0] == 0 and h.t[0] == 2.0 and h.t2[0] == 2.0


def test_duplicate_triangles_lowest_id(orc):
    rng = np.random.default_rng(4)
    tris = (rng.uniform(-5, 5, size=(10, 3, 3)) + 20.0).astype(np.float32)   # off the ray
    tris[7] = TRI
    tris[3] = TRI
    h = orc.closest_brute(tris, ray((1, 1, -100), (0, 0, 1))[None])
    assert h.id[0] == 3 and h.t[0] == 105.0


def test_t_interval_is_open(orc):
    tris = TRI[None]
    assert orc.closest_brute(tris, ray((1, 1, 0), (0, 0, 1), 0.0, 5.0)[None]).id[0] == -1
    assert orc.closest_brute(tris, ray((1, 1, 0), (0, 0, 1), 0.0, 5.0001)[None]).id[0] == 0
    assert orc.closest_brute(tris, ray((1, 1, 0), (0, 0, 1), 5.0, 9.0)[None]).id[0] == -1
    assert orc.closest_brute(tris, ray((1, 1, 0), (0, 0, 1), 4.999, 9.0)[None]).id[0] == 0


def test_invalid_rays_miss(orc):
    tris = TRI[None]
    bad = [ray((1, 1, 0), (0, 0, 1), 3.0, 3.0), ray((1, 1, 0), (0, 0, 1), 4.0, 1.0),
           ray((np.nan, 1, 0), (0, 0, 1)), ray((1, 1, 0), (0, np.inf, 1)),
           ray((1, 1, 0), (0, 0, 1), np.nan, 9.0), ray((1, 1, 0), (0, 0, 0))]
    h = orc.closest_brute(tris, np.stack(bad))
    assert (h.id == -1).all() and np.isinf(h.t).all()
    assert (orc.any_brute(tris, np.stack(bad)) == 0).all()


def test_skip_returns_next_hit(orc):
    tris = np.stack([TRI, TRI + np.float32([0, 0, 3])])
    r = ray((1, 1, 0), (0, 0, 1))[None]
    assert orc.closest_brute(tris, r).id[0] == 0
    h = orc.closest_brute(tris, r, skip=np.array([0], np.int32))
    assert h.id[0] == 1 and h.t[0] == 8.0


def test_any_equals_closest_below_tmax_and_monotone(orc):
    sc, rays, _ = scenes.workload_tiny()
    rays = rays.copy()
    rng = np.random.default_rng(5)
    rays[:, 7] = rng.uniform(1, 200, len(rays)).astype(np.float32)
    h = orc.closest_brute(sc.tris, rays)
    a = orc.any_brute(sc.tris, rays)
    assert (a == (h.id >= 0)).all()
    r2 = rays.copy()
    r2[:, 7] *= 0.5
    a2 = orc.any_brute(sc.tris, r2)
    assert (a2 <= a).all()          # a shorter range never creates a hit


# --------------------------------------------------------------- BVH
def test_eq2_worked_example_costs(orc):
    g = json.load(open(os.path.join(GOLDEN, "eq2_worked_example.json")))
    for c in g["candidates"]:
        for alpha in (1.0, 0.5, 0.0):
            got = orc.eq2_cost(c["box_A"], c["k_A"], c["box_B"], c["k_B"], g["box_C"], alpha, (0, 0, 0))
            want = alpha * c["sah"] + (1 - alpha) * c["d2"] + 1.0
            assert abs(got - want) < 1e-12


def test_eq2_worked_example_tree(orc):
    g = json.load(open(os.path.join(GOLDEN, "eq2_worked_example.json")))
    tris = np.asarray(g["tris"], np.float32)
    for alpha_s, i_best in g["best_split"].items():
        b = orc.Bvh(tris, alpha=float(alpha_s), source=(0, 0, 0), max_leaf=1)
        e = b.export()
        # size of the root's left subtree = the chosen split index
        def size(c):
            if c < 0:
                return int(e["leaf_count"][-1 - c])
            return size(e["child"][c][0]) + size(e["child"][c][1])
        assert size(e["child"][0][0]) == i_best, alpha_s
    for alpha_s, depth in g["depth_max_leaf_1"].items():
        assert orc.Bvh(tris, alpha=float(alpha_s), source=(0, 0, 0), max_leaf=1).info()["depth"] == depth


def _root_left_size(e):
    def size(c):
        if c < 0:
            return int(e["leaf_count"][-1 - c])
        return size(e["child"][c][0]) + size(e["child"][c][1])
    return size(e["child"][0][0])


def test_eq2_worked_example_scale_free_costs(orc):
    """Eq. 2 with the scale-free distance term (reading c2): the hand-derived
    d^2 * k_C / diag(C)^2 of each candidate."""
    g = json.load(open(os.path.join(GOLDEN, "eq2_worked_example.json")))
    n1 = g["dist_norm_1"]
    for c in g["candidates"]:
        term = n1["term"][str(c["i"])]
        assert abs(c["d2"] * n1["k_C"] / n1["diag2_C"] - term) < 1e-12
        for alpha in (1.0, 0.5, 0.4, 0.0):
            got = orc.eq2_cost(c["box_A"], c["k_A"], c["box_B"], c["k_B"], g["box_C"], alpha, (0, 0, 0), dist_norm=1)
            want = alpha * c["sah"] + (1 - alpha) * term + 1.0
            assert abs(got - want) < 1e-12


def test_eq2_worked_example_scale_free_split(orc):
    """The split the scale-free term picks flips between alpha = 0.4 and 0.5,
    where the raw m^2 term still splits off the nearest triangle."""
    g = json.load(open(os.path.join(GOLDEN, "eq2_worked_example.json")))
    tris = np.asarray(g["tris"], np.float32)
    for alpha_s, i_best in g["dist_norm_1"]["best_split"].items():
        b = orc.Bvh(tris, alpha=float(alpha_s), source=(0, 0, 0), max_leaf=1, dist_norm=1)
        assert _root_left_size(b.export()) == i_best, alpha_s
    raw = orc.Bvh(tris, alpha=0.5, source=(0, 0, 0), max_leaf=1, dist_norm=0)
    assert _root_left_size(raw.export()) == g["best_split"]["0.5"] == 1


def test_eq2_worked_example_count_weighted_costs(orc):
    """Eq. 2 with the count-weighted scale-free distance term (dist_norm = 2):
    the hand-derived (k_A d_A^2 + k_B d_B^2) / diag(C)^2 of each candidate, and
    with equal counts the same value as the scale-free term."""
    g = json.load(open(os.path.join(GOLDEN, "eq2_worked_example.json")))
    n2, n1 = g["dist_norm_2"], g["dist_norm_1"]
    for c in g["candidates"]:
        i = str(c["i"])
        assert abs(0.5 * (n2["dA2"][i] + n2["dB2"][i]) - c["d2"]) < 1e-12
        term = n2["term"][i]
        assert abs((c["k_A"] * n2["dA2"][i] + c["k_B"] * n2["dB2"][i]) / n1["diag2_C"] - term) < 1e-12
        for alpha in (1.0, 0.5, 0.2, 0.1, 0.0):
            got = orc.eq2_cost(c["box_A"], c["k_A"], c["box_B"], c["k_B"], g["box_C"], alpha, (0, 0, 0), dist_norm=2)
            want = alpha * c["sah"] + (1 - alpha) * term + 1.0
            assert abs(got - want) < 1e-12
            if c["k_A"] == c["k_B"]:
                same = orc.eq2_cost(c["box_A"], c["k_A"], c["box_B"], c["k_B"], g["box_C"], alpha, (0, 0, 0),
                                    dist_norm=1)
                assert abs(got - same) < 1e-12


def test_eq2_worked_example_count_weighted_split(orc):
    """The exact sweep with the count-weighted term picks the hand-derived
    root split on each side of its crossover (alpha = 0.1228...), and the
    lower of two equal-cost splits (i = 1 against i = 3) at alpha = 0."""
    g = json.load(open(os.path.join(GOLDEN, "eq2_worked_example.json")))
    tris = np.asarray(g["tris"], np.float32)
    for alpha_s, i_best in g["dist_norm_2"]["best_split"].items():
        b = orc.Bvh(tris, alpha=float(alpha_s), source=(0, 0, 0), max_leaf=1, dist_norm=2)
        assert _root_left_size(b.export()) == i_best, alpha_s


def test_tree_cost_alpha_half_worked_example(orc):
    """The recursive Eq. 2 tree cost at alpha = 0.5 (the recursion the quality
    bound of reading c6 uses) on the worked example, raw and scale-free: the
    hand-derived value for the hand-given tree, and the exact sweep builds
    exactly that tree."""
    g = json.load(open(os.path.join(GOLDEN, "eq2_worked_example.json")))
    tris = np.asarray(g["tris"], np.float32)
    tc = g["tree_cost_alpha_0.5"]
    for key, dn in (("raw", 0), ("scale_free", 1)):
        t = tc[key]
        child = np.asarray(t["child"], np.int32)
        lf = np.arange(4, dtype=np.int64)
        lc = np.ones(4, np.int64)
        prims = np.asarray([l[0] for l in t["leaves"]], np.int32)
        got = orc.tree_cost(tris, child, lf, lc, prims, 0.5, (0, 0, 0), dist_norm=dn)
        assert abs(got - t["cost"]) < 1e-12 * t["cost"], key
        b = orc.Bvh(tris, alpha=0.5, source=(0, 0, 0), max_leaf=1, dist_norm=dn)
        assert abs(b.cost() - t["cost"]) < 1e-12 * t["cost"], key
    # a slip in the recursion shows: the children's costs left out (k t_i used
    # instead) or the area ratio against the wrong box change the value
    t = tc["raw"]
    flat = 0.5 * ((2 / 14) * 1 + (10 / 14) * 3) + 0.5 * 10.5 + 1
    assert abs(flat - t["cost"]) > 1.0


def test_eq2_costs_scale_with_t_i_and_t_trav(orc):
    """Eq. 2 with t_i = 2.5 and t_trav = 0.75 on the worked example: the SAH
    term scales with t_i, so does the scale-free distance term (it carries
    k_C t_i), the raw m^2 term does not, and t_trav is added once."""
    g = json.load(open(os.path.join(GOLDEN, "eq2_worked_example.json")))
    n1 = g["dist_norm_1"]
    for c in g["candidates"]:
        for alpha in (1.0, 0.5, 0.0):
            for dn, term in ((0, c["d2"]), (1, n1["term"][str(c["i"])] * 2.5)):
                got = orc.eq2_cost(c["box_A"], c["k_A"], c["box_B"], c["k_B"], g["box_C"], alpha, (0, 0, 0),
                                   t_i=2.5, t_trav=0.75, dist_norm=dn)
                want = alpha * 2.5 * c["sah"] + (1 - alpha) * term + 0.75
                assert abs(got - want) < 1e-12, (c["i"], alpha, dn)


def test_t_i_weights_the_raw_split_and_t_trav_does_not(orc):
    """With the raw m^2 term at alpha = 0.5, t_i = 20 makes the SAH term win:
    costs 10 SAH + d^2/2 + t_trav = 29.11 / 26.39 / 36.11 for i = 1 / 2 / 3,
    so the balanced split i = 2 replaces i = 1 (t_i = 1).  t_trav is added to
    every candidate and never moves the split (reading c3)."""
    g = json.load(open(os.path.join(GOLDEN, "eq2_worked_example.json")))
    tris = np.asarray(g["tris"], np.float32)
    def left(**kw):
        return _root_left_size(orc.Bvh(tris, alpha=0.5, source=(0, 0, 0), max_leaf=1, **kw).export())
    assert left(t_i=1.0) == 1 and left(t_i=20.0) == 2
    assert left(t_i=1.0, t_trav=7.0) == 1 and left(t_i=20.0, t_trav=0.0) == 2


def _unit_tri(x, y):
    return [[x, y, 0.0], [x + 1.0, y, 0.0], [x, y + 1.0, 0.0]]


def _leaf_prims(e, c):
    assert c < 0
    k = -1 - c
    f, n = int(e["leaf_first"][k]), int(e["leaf_count"][k])
    return sorted(e["prims"][f:f + n].tolist())


def test_split_ties_go_to_the_lowest_axis(orc):
    """Four flat unit triangles on a 2 x 2 grid (ids 0..3 at (0,0), (2,0),
    (0,2), (2,2)), alpha = 1.  Cutting the grid along x or along y gives
    children of area 2*1*3 = 6 with 2 triangles each, SAH = 24/18 for both,
    from the same operands: an exact tie, which the reading breaks towards
    the lowest axis.  The x cut keeps {0, 2} together; the y cut would give
    {0, 1}."""
    tris = np.asarray([_unit_tri(0, 0), _unit_tri(2, 0), _unit_tri(0, 2), _unit_tri(2, 2)], np.float32)
    e = orc.Bvh(tris, alpha=1.0, source=(0, 0, 0), max_leaf=2).export()
    assert len(e["child"]) == 1
    assert _leaf_prims(e, e["child"][0][0]) == [0, 2] and _leaf_prims(e, e["child"][0][1]) == [1, 3]


def test_split_ties_go_to_the_lowest_split_index(orc):
    """Three flat unit triangles at x = 0, 2, 4 and the source at the centre
    of symmetry (2.5, 0.5, 0).  Splits after one and after two triangles are
    mirror images: SAH 2*1 + 6*2 against 6*2 + 2*1 (over 10), distance terms
    4 + 1 against 1 + 4, equal at every alpha; the reading takes the lower
    split index, so the left child holds triangle 0 alone."""
    tris = np.asarray([_unit_tri(0, 0), _unit_tri(2, 0), _unit_tri(4, 0)], np.float32)
    for alpha in (1.0, 0.5, 0.0):
        for dn in (0, 1):
            e = orc.Bvh(tris, alpha=alpha, source=(2.5, 0.5, 0.0), max_leaf=1, dist_norm=dn).export()
            assert _leaf_prims(e, e["child"][0][0]) == [0], (alpha, dn)


def test_split_candidates_follow_the_centroid_order_ties_by_id(orc):
    """Candidates are the prefixes of the triangles sorted by centroid on
    each axis, equal centroids in id order.  Triangles in planes x = const:
    t0 at (0,0,0), t1 at (0,5,5) (same x as t0), t2 at (10,10,10); raw
    distance term, alpha = 0, source at t1's box centre (0, 5.5, 5.5).
    Every axis then offers {t0}|{t1,t2} (d^2 = (50 + 37.5)/2, cost 44.75)
    and {t0,t1}|{t2} ((12.5 + 150)/2, cost 82.25), so t0 is split off.  The
    cheaper {t1}|{t0,t2} ((0 + 25)/2, cost 13.5) would be a candidate only
    if t1 came before t0 on x."""
    def tri(x, y, z):
        return [[x, y, z], [x, y + 1.0, z], [x, y, z + 1.0]]
    tris = np.asarray([tri(0, 0, 0), tri(0, 5, 5), tri(10, 10, 10)], np.float32)
    src = (0.0, 5.5, 5.5)
    c = orc.eq2_cost([0, 0, 0, 0, 1, 1], 1, [0, 5, 5, 10, 11, 11], 2, [0, 0, 0, 10, 11, 11], 0.0, src)
    assert c == 44.75
    e = orc.Bvh(tris, alpha=0.0, source=src, max_leaf=1).export()
    assert _leaf_prims(e, e["child"][0][0]) == [0]


def _check_structure(orc, tris, b, max_leaf):
    e = b.export()
    assert sorted(e["prims"].tolist()) == list(range(len(tris)))
    assert (e["leaf_count"] >= 1).all() and (e["leaf_count"] <= max_leaf).all()
    cnt = e["leaf_count"].sum()
    assert cnt == len(tris)
    child = e["child"]
    if len(child):
        refs = child.reshape(-1)
        internal = refs[refs >= 0]
        assert sorted(internal.tolist()) == list(range(1, len(child)))   # each non-root once
        assert sorted((-1 - refs[refs < 0]).tolist()) == list(range(len(e["leaf_first"])))


@pytest.mark.parametrize("alpha", [1.0, 0.7, 0.4, 0.0])
@pytest.mark.parametrize("max_leaf", [1, 4, 250, 820])
def test_bvh_equals_brute_tiny_city(orc, alpha, max_leaf):
    sc, rays, _ = scenes.workload_tiny()
    ref = orc.closest_brute(sc.tris, rays)
    ref_any = orc.any_brute(sc.tris, rays)
    for dn in (0, 1, 2):
        b = orc.Bvh(sc.tris, alpha=alpha, source=sc.tx[0], max_leaf=max_leaf, dist_norm=dn)
        _check_structure(orc, sc.tris, b, max_leaf)
        h = b.closest(rays)
        assert (h.id == ref.id).all()
        assert np.array_equal(h.t, ref.t) and np.array_equal(h.t2, ref.t2)
        assert np.array_equal(h.u, ref.u) and np.array_equal(h.v, ref.v)
        assert (b.any(rays) == ref_any).all()


@pytest.mark.parametrize("alpha,dn", [(1.0, 0), (0.7, 1), (0.4, 1), (0.0, 0)])
def test_bvh_equals_brute_medium_city_sample(orc, alpha, dn):
    sc, rays, _ = scenes.workload_medium(level=5)
    rnd = scenes.random_rays(sc, 1500, seed=11, tmax=400.0)
    allr = np.concatenate([rays, rnd])
    ref = orc.closest_brute(sc.tris, allr)
    b = orc.Bvh(sc.tris, alpha=alpha, source=sc.tx[0], max_leaf=4, dist_norm=dn)
    h = b.closest(allr)
    assert (h.id == ref.id).all() and np.array_equal(h.t, ref.t) and np.array_equal(h.t2, ref.t2)
    assert (b.any(allr) == (ref.id >= 0)).all()


def test_bvh_grazing_and_skip_equal_brute(orc):
    # rays aimed exactly at building vertices and edge midpoints, plus skips
    sc = scenes.tiny_city(seed=1)
    v = sc.tris.reshape(-1, 3).astype(np.float64)
    rng = np.random.default_rng(6)
    pick = rng.choice(len(v), 1500)
    tgt = np.concatenate([v[pick], 0.5 * (v[pick] + v[rng.choice(len(v), 1500)])])
    o = np.array([100.0, 100.0, 30.0])
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = scenes.make_rays(o, d, 0.0, 1e4)
    skip = rng.integers(-1, sc.n_tri, len(rays)).astype(np.int32)
    ref = orc.closest_brute(sc.tris, rays, skip=skip)
    for alpha in (1.0, 0.4):
        b = orc.Bvh(sc.tris, alpha=alpha, source=o, max_leaf=2)
        h = b.closest(rays, skip=skip)
        assert (h.id == ref.id).all() and np.array_equal(h.t, ref.t)


def test_alpha1_tree_cost_is_textbook_sah(orc):
    """At alpha = 1 the recursive Eq. 2 tree cost equals the textbook SAH sum
    sum_internal S(n)/S(root) t_trav + sum_leaves S(l)/S(root) k_l t_i."""
    sc = scenes.tiny_city(seed=1)
    b = orc.Bvh(sc.tris, alpha=1.0, source=(0, 0, 0), max_leaf=4)
    e = b.export()
    tb = sc.tris.astype(np.float64)

    def box_of(ids):
        p = tb[ids].reshape(-1, 3)
        return p.min(0), p.max(0)

    def area(lo, hi):
        dx, dy, dz = hi - lo
        return 2 * (dx * dy + dy * dz + dz * dx)

    def gather(c):
        if c < 0:
            l = -1 - c
            return list(e["prims"][e["leaf_first"][l]: e["leaf_first"][l] + e["leaf_count"][l]])
        return gather(e["child"][c][0]) + gather(e["child"][c][1])

    s_root = area(*box_of(list(range(sc.n_tri))))
    total = 0.0
    for i in range(len(e["child"])):
        total += area(*box_of(gather(i))) / s_root * 1.0
    for l in range(len(e["leaf_first"])):
        ids = e["prims"][e["leaf_first"][l]: e["leaf_first"][l] + e["leaf_count"][l]]
        total += area(*box_of(ids)) / s_root * len(ids)
    assert abs(b.cost() - total) < 1e-9 * total


def test_alpha1_separates_two_clusters(orc):
    rng = np.random.default_rng(7)
    a = rng.uniform(0, 1, size=(20, 3, 3))
    b = rng.uniform(0, 1, size=(20, 3, 3)) + np.array([50.0, 0, 0])
    tris = np.concatenate([a, b]).astype(np.float32)
    perm = rng.permutation(40)
    tris = tris[perm]
    t = orc.Bvh(tris, alpha=1.0, max_leaf=4)
    e = t.export()

    def gather(c):
        if c < 0:
            l = -1 - c
            return list(e["prims"][e["leaf_first"][l]: e["leaf_first"][l] + e["leaf_count"][l]])
        return gather(e["child"][c][0]) + gather(e["child"][c][1])

    left = np.array(gather(e["child"][0][0]))
    side = perm[left] >= 20
    assert side.all() or (~side).all()
    assert len(left) == 20


# --------------------------------------------------------------- reflection
def test_ground_reflection_image_method(orc):
    A = 500.0
    tris = np.asarray(scenes._ground(0, 0, A, A), np.float32)
    tx = np.array([200.0, 240.0, 30.0])
    rng = np.random.default_rng(8)
    g = np.stack([rng.uniform(10, 490, 500), rng.uniform(10, 490, 500), np.zeros(500)], 1)
    d = g - tx
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = scenes.make_rays(tx, d, 0.0, 2000.0)
    h = orc.closest_brute(tris, rays)
    assert (h.id >= 0).all()
    out = orc.reflect(tris, rays, h.id, h.t)
    image = np.array([tx[0], tx[1], -tx[2]])
    want = out[:, 0:3] - image
    want /= np.linalg.norm(want, axis=1, keepdims=True)
    dr = out[:, 4:7]
    d32 = rays[:, 4:7].astype(np.float64)
    assert np.allclose(np.linalg.norm(dr, axis=1), np.linalg.norm(d32, axis=1), rtol=1e-14)
    assert np.allclose(dr / np.linalg.norm(dr, axis=1, keepdims=True), want, atol=1e-6)
    assert np.allclose(out[:, 2], 0.0, atol=1e-9)
    # angle of incidence equals angle of reflection (normal +-z)
    assert np.allclose(np.abs(dr[:, 2]), np.abs(d32[:, 2]), rtol=1e-14)
    assert np.allclose(out[:, 7], 2000.0 - h.t, rtol=0, atol=1e-9)
    assert (out[:, 3] == 0).all()


def test_wall_reflection_flips_normal_component(orc):
    wall = np.array([[[10, -50, -50], [10, 50, -50], [10, 0, 50]]], np.float32)
    rng = np.random.default_rng(9)
    d = rng.normal(size=(200, 3))
    d[:, 0] = np.abs(d[:, 0]) + 0.2
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = scenes.make_rays((0, 0, 0), d * 0.25, 0.0, 1e3)
    h = orc.closest_brute(wall, rays)
    ok = h.id >= 0
    assert ok.sum() > 100
    out = orc.reflect(wall, rays[ok], h.id[ok], h.t[ok])
    d32 = rays[ok][:, 4:7].astype(np.float64)
    assert np.allclose(out[:, 4], -d32[:, 0], rtol=1e-14)
    assert np.allclose(out[:, 5:7], d32[:, 1:3], rtol=1e-14)
    assert np.allclose(out[:, 0], 10.0, atol=1e-12)


# --------------------------------------------------------------- launch directions
@pytest.mark.parametrize("level", [0, 1, 2, 3, 5])
def test_icosphere_count_norm_and_symmetry(orc, level):
    f = 2 ** level
    p = orc.icosphere(level)
    assert p.shape == (10 * f * f + 2, 3)
    assert np.allclose(np.linalg.norm(p, axis=1), 1.0, atol=1e-15)
    key = lambda a: a[np.lexsort(np.round(a, 9).T)]
    for m in (np.diag([-1.0, 1, 1]), np.diag([1.0, -1, 1]), np.diag([1.0, 1, -1]),
              np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], float)):
        assert np.allclose(key(p @ m.T), key(p), atol=1e-12)
    assert np.allclose(p, scenes.icosphere_directions(level), atol=1e-15)
    # distinct points
    assert len(np.unique(np.round(p, 9), axis=0)) == len(p)


def test_icosphere_neighbour_angle():
    # the icosahedron's edge subtends atan(2) = 63.435 deg; a level-L grid spaces its
    # points about atan(2)/2^L apart (projection distortion stays within 25%)
    for level in (3, 4):
        p = scenes.icosphere_directions(level)
        c = p @ p.T
        np.fill_diagonal(c, -1)
        nn = np.degrees(np.arccos(np.clip(c.max(1), -1, 1)))
        expect = math.degrees(math.atan(2.0)) / 2 ** level
        assert 0.75 * expect < np.median(nn) < 1.25 * expect
        assert nn.min() > 0.5 * expect


def test_icosphere_base_vertices(orc):
    p = orc.icosphere(0)
    g = (1 + math.sqrt(5)) / 2
    n = math.sqrt(1 + g * g)
    vals = np.sort(np.abs(p).reshape(-1))
    assert np.allclose(vals[:12], 0.0) and np.allclose(vals[12:24], 1 / n) and np.allclose(vals[24:], g / n)


def test_fibonacci(orc):
    n = 4096
    p = orc.fibonacci(n)
    assert np.allclose(np.linalg.norm(p, axis=1), 1.0, atol=1e-15)
    assert np.allclose(p, scenes.fibonacci_directions(n), atol=1e-15)
    assert np.allclose(np.diff(p[:, 2]), -2.0 / n)          # equal-area bands
    assert np.abs(p.mean(0)).max() < 1e-3                   # balanced over the sphere


# --------------------------------------------------------------- generators
def test_generators_deterministic_and_counts():
    a = scenes.tiny_city(seed=1)
    b = scenes.tiny_city(seed=1)
    assert a.tris.tobytes() == b.tris.tobytes() and a.n_tri == 770
    m = scenes.medium_city(seed=2)
    assert m.tris.tobytes() == scenes.medium_city(seed=2).tris.tobytes()
    assert 17000 < m.n_tri < 23000
    # every prism contributes 4n - 4 triangles (walls 2n, caps 2(n-2))
    assert (m.n_tri - 2) % 4 == 0
    tx = m.tx[0]
    # the transmitter is not inside any building footprint's bounding circle
    assert tx[2] == 30.0


def test_metro_generator_counts_prisms_and_determinism():
    a = scenes.metro_city(n_buildings=300, size=1500.0)
    b = scenes.metro_city(n_buildings=300, size=1500.0)
    assert a.tris.tobytes() == b.tris.tobytes()
    # every building is a closed convex 8..16-gon prism: 4n - 4 triangles, plus 2 ground
    assert (a.n_tri - 2) % 4 == 0 and 300 * 28 <= a.n_tri - 2 <= 300 * 60
    # the first building, rebuilt with the per-prism generator from its own footprint
    t = a.tris.astype(np.float64)
    h = t[:, :, 2].max(axis=1)
    k = 0
    while t[k, 0, 2] == 0.0:  # building 0's walls start at its floor; its roof fan starts at z = h
        k += 1
    n = k // 2
    poly = t[0:2 * n:2, 0, :2]
    ref = np.asarray(scenes._prism(poly, h[0]), np.float64).astype(np.float32)
    assert np.array_equal(a.tris[:len(ref)], ref)


# --------------------------------------------------------------- reception (Sec. III.C, Eq. 4)
def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def test_receive_sphere_radius_closed_form(orc):
    # Eq. 4: r = l delta / sqrt(3).  A ray from the origin along a skew unit
    # direction; receivers at path length L, offset sideways by 0.99 r / 1.01 r
    d = _unit((3.0, -2.0, 1.5))
    side = _unit(np.cross(d, (0.0, 0.0, 1.0)))
    delta, L = 0.004, 200.0
    r = L * delta / math.sqrt(3.0)
    assert abs(r - 0.46188) < 1e-5  # 200 * 0.004 / 1.7320508
    rays = np.array([[0, 0, 0, 0, *d, 500.0]], np.float32)
    rx = np.array([L * d + 0.99 * r * side, L * d + 1.01 * r * side, L * d - 0.5 * r * side, L * d],
                  np.float32)
    pairs, vals = orc.receive(rays, np.array([np.inf], np.float32), rx, delta, 500.0)
    got = {int(j): (int(c), v) for (_, j, c), v in zip(pairs, vals)}
    assert set(got) == {0, 2, 3}
    for j in (0, 2, 3):
        assert got[j][0] == 1
        assert abs(got[j][1][0] - L) < 1e-4 and abs(got[j][1][2] - r) < 1e-6
    assert abs(got[3][1][1]) < 1e-4 and abs(got[0][1][1] - 0.99 * r) < 1e-4


def test_receive_segment_ends_and_hit_cut(orc):
    d = _unit((1.0, 1.0, 0.0))
    rays = np.array([[10, 20, 5, 30.0, *d, 400.0]], np.float32)  # segment starts at t = 30
    o = np.array([10.0, 20.0, 5.0])
    rx = np.array([o + 20 * d, o + 80 * d, o + 160 * d, o + 450 * d], np.float32)
    # no hit: [30, 400) -> 80 and 160 received, 20 (before tmin) and 450 (past tmax) not
    pairs, _ = orc.receive(rays, np.array([np.inf], np.float32), rx, 0.01, 400.0)
    assert sorted(int(j) for _, j, c in pairs if c == 1) == [1, 2]
    # a hit at t = 120 cuts the segment: only 80 remains
    pairs, _ = orc.receive(rays, np.array([120.0], np.float32), rx, 0.01, 400.0)
    assert sorted(int(j) for _, j, c in pairs if c == 1) == [1]


def test_receive_path_length_after_ground_bounce_is_image_distance(orc):
    # Tx at height h; a ray hits the ground plane z = 0 and reflects.  Along the
    # reflected ray the unfolded path length equals the distance from the
    # receiver to the mirror image of the Tx (image method), so Eq. 4 uses it.
    h, R0 = 30.0, 500.0
    tx = np.array([100.0, 50.0, h])
    g = np.array([160.0, 90.0, 0.0])
    d0 = _unit(g - tx)
    ground = np.array([[[-1e4, -1e4, 0], [3e4, -1e4, 0], [-1e4, 3e4, 0]]], np.float32)
    r0 = np.array([[*tx, 0.0, *d0, R0]], np.float32)
    hit = orc.closest_brute(ground, r0)
    assert hit.id[0] == 0
    refl = orc.reflect(ground, r0, hit.id, hit.t)
    r1 = refl.astype(np.float32)
    assert abs(refl[0, 7] - (R0 - np.linalg.norm(g - tx))) < 1e-4  # float32 direction
    image = tx * np.array([1, 1, -1])
    p = refl[0, :3] + 75.0 * refl[0, 4:7]  # a receiver on the reflected ray
    pairs, vals = orc.receive(r1, np.array([np.inf], np.float32), p[None].astype(np.float32), 0.01, R0)
    assert len(pairs) == 1 and pairs[0, 2] == 1
    assert abs(vals[0, 0] - np.linalg.norm(p - image)) < 1e-3


def test_receive_matches_cross_product_formula(orc):
    # the same rule written another way (numpy, float64): distance to the line
    # by |q x d| / |d|, foot by q.d / d.d; decisions agree outside the
    # tolerance band, whose pairs the checker marks as class 2
    rng = np.random.default_rng(7)
    n, m = 300, 200
    o = rng.uniform(-50, 50, (n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tmin = rng.uniform(0, 5, n)
    tmax = rng.uniform(50, 120, n)
    rays = np.concatenate([o, tmin[:, None], d, tmax[:, None]], 1).astype(np.float32)
    ht = np.where(rng.random(n) < 0.5, rng.uniform(10, 150, n), np.inf).astype(np.float32)
    rx = rng.uniform(-60, 60, (m, 3)).astype(np.float32)
    delta, R0, tol = 0.05, 150.0, 1e-6
    pairs, _ = orc.receive(rays, ht, rx, delta, R0, tol=tol)
    sure = {(int(i), int(j)) for i, j, c in pairs if c == 1}
    near = {(int(i), int(j)) for i, j, c in pairs}
    R = rays.astype(np.float64)
    P = rx.astype(np.float64)
    want = set()
    for i in range(n):
        oo, dd = R[i, :3], R[i, 4:7]
        q = P - oo
        ts = q @ dd / (dd @ dd)
        dist = np.linalg.norm(np.cross(q, dd), axis=1) / np.linalg.norm(dd)
        tend = min(float(ht[i]), R[i, 7])
        ok = (ts >= R[i, 3]) & (ts < tend) & (dist <= (R0 - R[i, 7] + ts) * delta / math.sqrt(3))
        want |= {(i, int(j)) for j in np.nonzero(ok)[0]}
    assert len(want) > 20
    assert sure <= want <= near


# --------------------------------------------------------------- ray action range (Sec. II.B)
def _box_dist(tris, s):
    lo = tris.min(axis=1).astype(np.float64)
    hi = tris.max(axis=1).astype(np.float64)
    d = np.maximum(np.maximum(lo - s, s - hi), 0.0)
    return np.sqrt((d * d).sum(1))


def test_range_pruning_keeps_every_triangle_a_bounce_chain_hits(orc):
    # a path of total length <= R never reaches a point farther than R from
    # its source (triangle inequality), so pruning the triangles whose box is
    # farther than R drops no hit at any order: check on bounce chains
    sc = scenes.medium_city(seed=2)
    src = np.array(sc.tx[0], np.float64)
    R = 180.0
    rays = scenes.make_rays(src, scenes.fibonacci_directions(3000), 0.0, R)
    skip = None
    dist = _box_dist(sc.tris, src)
    hit_any = 0
    for order in range(3):
        h = orc.closest_brute(sc.tris, rays, skip=skip)
        ok = h.id >= 0
        hit_any += ok.sum()
        assert (dist[h.id[ok]] <= R * (1 + 1e-9)).all()
        nxt = orc.reflect(sc.tris, rays, h.id, h.t)
        keep = ok & (nxt[:, 7] > 0)
        rays = nxt[keep].astype(np.float32)
        skip = h.id[keep]
        if len(rays) == 0:
            break
    assert hit_any > 1000
