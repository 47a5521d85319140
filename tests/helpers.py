"""Shared test helpers: comparison of GPU hits with the float64 checker."""
import numpy as np

T_REL = 1e-5     # hit distance tolerance, relative
T_ABS = 1e-6     # absolute floor for t -> 0 (metres)
TIE_REL = 1e-6   # rays whose two nearest hits are this close are near-ties


def split_hits(h):
    h = np.ascontiguousarray(h, dtype=np.float32)
    return h[:, 0].astype(np.float64), h.view(np.int32)[:, 1].copy(), h[:, 2], h[:, 3]


def compare_closest(gpu_hits, ref, tris=None, rays=None, label=""):
    """Assert the tolerance contract; returns (n_rays, n_hits, n_near_ties).

    ids must match bit for bit except on near-tie rays (two nearest oracle
    distances within 1e-6 relative); there the GPU id must be a triangle the
    ray really hits at the reported distance.  t within 1e-5 t + 1e-6.
    """
    t, ids, u, v = split_hits(gpu_hits)
    n = len(ids)
    rt, rid = ref.t, ref.id
    with np.errstate(invalid="ignore"):  # inf - inf on rays without a second hit
        tie = np.isfinite(ref.t2) & (ref.t2 - rt <= TIE_REL * np.abs(rt))
    bad_id = (ids != rid) & ~tie
    if bad_id.any():
        k = np.nonzero(bad_id)[0][:10]
        raise AssertionError("%s: %d id mismatches, first rays %s gpu %s ref %s t_gpu %s t_ref %s t2_ref %s" % (
            label, bad_id.sum(), k, ids[k], rid[k], t[k], rt[k], ref.t2[k]))
    miss = rid < 0
    assert (ids[miss] == -1).all() and np.isinf(t[miss]).all(), label
    hit = ~miss
    err = np.abs(t[hit] - rt[hit])
    lim = T_REL * rt[hit] + T_ABS
    if not (err <= lim).all():
        k = np.nonzero(hit)[0][err > lim][:10]
        raise AssertionError("%s: t out of tolerance on rays %s: gpu %s ref %s" % (label, k, t[k], rt[k]))
    if tie.any() and tris is not None and rays is not None:
        import oracle
        for k in np.nonzero(tie & (ids != rid))[0][:200]:
            ok, tt, _, _ = oracle.tri_hit(tris[ids[k]], rays[k])
            assert ok and abs(tt - rt[k]) <= T_REL * rt[k] + T_ABS, (label, k)
    return n, int(hit.sum()), int(tie.sum())


def fibonacci_launch_perm(n):
    """Spiral index held by each slot of an n-ray Fibonacci launch in band
    order, by brute force: the spiral is cut into bands of w consecutive
    points, w the largest of the Fibonacci numbers 2, 3, 5, 8, ... with
    w^2 <= 80 n; the slots of each full band take its points in increasing
    azimuth measured from the band's first point (azimuth of point i:
    i (3 - sqrt 5) / 2 turns); the slots after the last full band keep their
    own point."""
    a, w = 1, 2
    while (a + w) ** 2 <= 80 * n:
        a, w = w, a + w
    g = (3.0 - np.sqrt(5.0)) / 2.0
    j = np.arange(w, dtype=np.float64)
    order = np.argsort(np.mod(j * g, 1.0), kind="stable")
    perm = np.arange(n, dtype=np.int64)
    for b in range(n // w):
        perm[b * w:(b + 1) * w] = b * w + order
    return perm

