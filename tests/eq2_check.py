"""Split-by-split check of a device-built BVH against Eq. 2 (Sec. II.B, Eq. 2;
Sec. II.C, Fig. 2), scored by the float64 checker.

The device does not sweep every object split (reading c6).  Its candidate
set at a node of n records is:

* n > 32 (big-node chunks, CTA splits, warp splits in global memory): for each
  axis, `bins` equal slabs of the node's centroid interval [cmin, cmax]; the
  candidate at plane p (1 <= p < bins) sends left the records whose slab index
  is below p.  Centre = (lo + hi) * 0.5 of the triangle's box, slab index =
  trunc((c - cmin) * scale) clamped to [0, bins - 1], scale = bins (1 - 1e-6) /
  (cmax - cmin), all in float32.  Float32 decides these integers on the
  device, so the same float32 operations decide them here.
* n <= 32: the n - 1 prefix splits of the node's records in the order of
  their 30-bit Morton keys (ties: lower triangle id); that order is the node's
  leaf order, which the export returns.

For every internal node the check rebuilds that candidate set from the
triangles, scores every candidate with ``oracle.eq2_cost`` on the exact child
boxes and counts, and requires the device's split to be a minimum within the
float32 error of the device's cost evaluation (stated in ``cost_tol``).
"""
from __future__ import annotations

import numpy as np

MICRO = 32
U32 = 2.0 ** -24
F32 = np.float32
ONE_MINUS = F32(1.0) - F32(1e-6)


def tri_boxes(tris):
    t = np.asarray(tris, np.float32).reshape(-1, 3, 3)
    return t.min(axis=1), t.max(axis=1)


def centres32(lo, hi):
    """Box centres (lo + hi) * 0.5 in float32."""
    return ((lo + hi).astype(F32) * F32(0.5)).astype(F32)


def slab_index(c, K):
    """Slab index of every centre coordinate c (one axis) on the node's own interval."""
    c = np.asarray(c, F32)
    cmin, cmax = c.min(), c.max()
    ext = F32(cmax - cmin)
    scale = F32(F32(F32(K) * ONE_MINUS) / ext) if ext > 0 else F32(0.0)
    b = np.trunc((F32(c - cmin) * scale).astype(F32)).astype(np.int64)
    return np.clip(b, 0, K - 1)


def morton_keys(lo, hi):
    """30-bit Morton keys of the box centres on the scene's centroid box."""
    c = centres32(lo, hi)
    cl, ch = c.min(axis=0), c.max(axis=0)
    q = np.zeros(c.shape, np.int64)
    for a in range(3):
        ext = F32(ch[a] - cl[a])
        msc = F32(F32(1023.99) / ext) if ext > 0 else F32(0.0)
        q[:, a] = np.clip(np.trunc((F32(c[:, a] - cl[a]) * msc).astype(F32)), 0, 1023).astype(np.int64)

    def spread(v):
        out = np.zeros_like(v)
        for bit in range(10):
            out |= ((v >> bit) & 1) << (3 * bit)
        return out

    return (spread(q[:, 0]) << 2) | (spread(q[:, 1]) << 1) | spread(q[:, 2])


def node_ranges(ex):
    """(first, n, nl) of every internal node: its records are prims[first:first+n],
    the left child's the first nl of them.  Asserts that every subtree is contiguous."""
    child, lf, lc = ex["child"], ex["leaf_first"], ex["leaf_count"]
    m = len(child)
    first = np.full(m, -1, np.int64)
    cnt = np.zeros(m, np.int64)
    nl = np.zeros(m, np.int64)
    order = []
    st = [0] if m else []
    seen = np.zeros(m, bool)
    while st:  # pre-order, then resolve in reverse (children before parents)
        x = st.pop()
        assert not seen[x], "node %d reached twice" % x
        seen[x] = True
        order.append(x)
        for c in child[x]:
            if c >= 0:
                st.append(int(c))
    assert seen.all(), "unreachable internal nodes"
    for x in reversed(order):
        rng = []
        for c in child[x]:
            if c >= 0:
                rng.append((first[c], cnt[c]))
            else:
                l = -1 - int(c)
                rng.append((int(lf[l]), int(lc[l])))
        (fa, na), (fb, nb) = rng
        assert fb == fa + na, "node %d: children not contiguous" % x
        first[x], cnt[x], nl[x] = fa, na + nb, na
    return first, cnt, nl


def cost_tol(sah_abs, term_abs, dA, dB, M, alpha, w, t_trav):
    """Float32 error bound of the device's Eq. 2 value of one candidate: 32 unit
    roundoffs of every term (areas, products, fast reciprocals), plus the
    rounding of the box centres against the source (each centre coordinate off
    by at most 2 u M, M the largest coordinate of the node box and the source)."""
    rel = 32.0 * U32 * (alpha * sah_abs + (1.0 - alpha) * term_abs + abs(t_trav))
    dist = (1.0 - alpha) * w * (dA + dB) * 8.0 * U32 * M
    return rel + dist


class Checker:
    """Scores candidates of one tree with the checker's Eq. 2."""

    def __init__(self, orc, tris, alpha, source, dist_norm=0, t_i=1.0, t_trav=1.0, bins=16):
        self.orc = orc
        self.lo, self.hi = tri_boxes(tris)
        self.alpha, self.t_i, self.t_trav = float(alpha), float(t_i), float(t_trav)
        # the device holds the build parameters as float32
        self.src = np.asarray(source, np.float32).astype(np.float64)
        self.alpha = float(F32(alpha))
        self.dist_norm = int(dist_norm)
        self.K = int(bins)

    def score(self, la, ha, ka, lb, hb, kb):
        """(cost, tolerance) of the candidate with children boxes A=[la,ha], B=[lb,hb]."""
        lc, hc = np.minimum(la, lb), np.maximum(ha, hb)
        ba = np.concatenate([la, ha]).astype(np.float64)
        bb = np.concatenate([lb, hb]).astype(np.float64)
        bc = np.concatenate([lc, hc]).astype(np.float64)
        c = self.orc.eq2_cost(ba, ka, bb, kb, bc, self.alpha, self.src, t_i=self.t_i, t_trav=self.t_trav,
                              dist_norm=self.dist_norm)
        # magnitudes for the tolerance (float64, no part of the cost itself)
        def area(lo, hi):
            d = (hi - lo).astype(np.float64)
            return 2.0 * (d[0] * d[1] + d[1] * d[2] + d[2] * d[0])
        sc = area(lc, hc)
        sah = (area(la, ha) * ka + area(lb, hb) * kb) / sc * self.t_i if sc > 0 else (ka + kb) * self.t_i
        dA = float(np.linalg.norm(0.5 * (la.astype(np.float64) + ha) - self.src))
        dB = float(np.linalg.norm(0.5 * (lb.astype(np.float64) + hb) - self.src))
        w = 1.0
        term = 0.5 * (dA * dA + dB * dB)
        if self.dist_norm:
            diag2 = float(((hc - lc).astype(np.float64) ** 2).sum())
            if self.dist_norm == 2:
                # (ka dA^2 + kb dB^2) t_i / diag2: a centre error moves it by at most
                # 2 max(ka, kb) t_i / diag2 (dA + dB) times the error
                term = (ka * dA * dA + kb * dB * dB) * self.t_i / diag2 if diag2 > 0 else 0.0
                w = 2.0 * max(ka, kb) * self.t_i / diag2 if diag2 > 0 else 0.0
            else:
                w = (ka + kb) * self.t_i / diag2 if diag2 > 0 else 0.0
                term *= w
        M = max(float(np.abs(np.concatenate([lc, hc])).max()), float(np.abs(self.src).max()))
        return c, cost_tol(abs(sah), abs(term), dA, dB, M, self.alpha, w, self.t_trav)

    def prefix_candidates(self, ids):
        """All prefix splits of the records `ids` in the given order: list of (nl, cost, tol)."""
        lo, hi = self.lo[ids], self.hi[ids]
        pl, ph = np.minimum.accumulate(lo), np.maximum.accumulate(hi)
        sl, sh = np.minimum.accumulate(lo[::-1])[::-1], np.maximum.accumulate(hi[::-1])[::-1]
        n = len(ids)
        out = []
        for q in range(1, n):
            c, t = self.score(pl[q - 1], ph[q - 1], q, sl[q], sh[q], n - q)
            out.append((q, c, t))
        return out

    def binned_candidates(self, ids):
        """Binned candidates of a node > 32 records: list of ((axis, plane), left mask, cost, tol);
        planes that leave one side empty, or repeat the set of the plane before, are skipped."""
        lo, hi = self.lo[ids], self.hi[ids]
        c = centres32(lo, hi)
        n = len(ids)
        out = []
        for a in range(3):
            b = slab_index(c[:, a], self.K)
            prev = -1
            for p in range(1, self.K):
                left = b < p
                k = int(left.sum())
                if k == 0 or k == n or k == prev:
                    prev = k
                    continue
                prev = k
                cost, tol = self.score(lo[left].min(0), hi[left].max(0), k, lo[~left].min(0), hi[~left].max(0),
                                       n - k)
                out.append(((a, p), left, cost, tol))
        return out


def check_tree(orc, tris, ex, alpha, source, dist_norm, bins, t_i=1.0, t_trav=1.0, sample=None, seed=0):
    """Assert that every split of the exported tree is an Eq. 2 minimum over the
    device's candidates.  sample: check every node of more than 1024 records and
    this many of the others, drawn with `seed` (None: every node).  Returns
    per-path counts and the worst relative gap."""
    chk = Checker(orc, tris, alpha, source, dist_norm=dist_norm, t_i=t_i, t_trav=t_trav, bins=bins)
    prims = ex["prims"]
    first, cnt, nl = node_ranges(ex)
    keys = morton_keys(chk.lo, chk.hi)
    child = ex["child"]
    parent_n = np.full(len(child), 1 << 62, np.int64)
    for x in range(len(child)):
        for s in range(2):
            if child[x][s] >= 0:
                parent_n[child[x][s]] = cnt[x]
    stats = dict(binned=0, binned_exact=0, micro=0, micro_exact=0, middle=0, micro_roots=0, worst_gap=0.0,
                 over_1024=0, cta_range=0)
    todo = np.arange(len(child))
    if sample is not None:
        big = todo[cnt > 1024]
        rest = todo[cnt <= 1024]
        pick = np.random.default_rng(seed).choice(rest, min(int(sample), len(rest)), replace=False)
        todo = np.sort(np.concatenate([big, pick]))
    for x in todo:
        ids = prims[first[x]: first[x] + cnt[x]]
        n = len(ids)
        if n <= MICRO:
            if parent_n[x] > MICRO:  # the root of a small subtree: its leaf order is the Morton order
                kk = keys[ids]
                order = np.lexsort((ids, kk))
                assert np.array_equal(order, np.arange(n)), "node %d: records not in (Morton key, id) order" % x
                stats["micro_roots"] += 1
            cands = chk.prefix_candidates(ids)
            mine = [c for c in cands if c[0] == nl[x]]
            assert len(mine) == 1
            _, c_dev, t_dev = mine[0]
            best = min(cands, key=lambda c: c[1])
            stats["micro"] += 1
            stats["micro_exact"] += int(best[0] == nl[x])
        else:
            cands = chk.binned_candidates(ids)
            left_ids = np.zeros(n, bool)
            left_ids[: nl[x]] = True  # the left child's records come first in leaf order
            if not cands:
                # no plane separates anything: the device halves the range
                assert nl[x] == n // 2, "node %d: no candidate, yet not split in the middle" % x
                stats["middle"] += 1
                continue
            mine = [c for c in cands if np.array_equal(c[1], left_ids)]
            assert mine, "node %d (n=%d, nl=%d): the device's split is not one of its candidates" % (x, n, nl[x])
            _, _, c_dev, t_dev = mine[0]
            best = min(cands, key=lambda c: c[2])
            stats["binned"] += 1
            stats["over_1024" if n > 1024 else "cta_range"] += 1
            stats["binned_exact"] += int(np.array_equal(best[1], left_ids))
            best = (None, best[2], best[3])
        gap = c_dev - best[1]
        assert gap <= t_dev + best[2], (
            "node %d (n=%d): device split costs %.9g, the minimum over its candidates %.9g (tolerance %.3g)" % (
                x, n, c_dev, best[1], t_dev + best[2]))
        stats["worst_gap"] = max(stats["worst_gap"], gap / max(abs(best[1]), 1e-30))
    return stats
