"""CPU test of the split-by-split Eq. 2 check (tests/eq2_check.py) used on
device-built trees: a tree built in Python by the same candidate rule, taking
the checker's Eq. 2 minimum at every node, passes it; trees built with a
planted mistake in the cost (a mirrored source, the distance term without its
normalisation, the SAH tree checked as an alpha < 1 tree) fail it."""
import numpy as np
import pytest

from paper_2208_10008_gb300 import scenes
import eq2_check as E


def _build(orc, tris, alpha, source, dist_norm, bins, max_leaf):
    """Top-down build (Sec. II.C, Fig. 2) with the device's candidate sets and the
    checker's Eq. 2 as the split rule; returns the tree in the export form."""
    chk = E.Checker(orc, tris, alpha, source, dist_norm=dist_norm, bins=bins)
    keys = E.morton_keys(chk.lo, chk.hi)
    child, leaves, prims = [], [], []

    def leaf(ids):
        leaves.append((len(prims), len(ids)))
        prims.extend(int(i) for i in ids)
        return -len(leaves)   # -1 - leaf index

    def rec(ids, sorted_small):
        n = len(ids)
        if n <= max_leaf:
            return leaf(ids)
        if n <= E.MICRO and not sorted_small:
            ids = ids[np.lexsort((ids, keys[ids]))]
            sorted_small = True
        me = len(child)
        child.append([0, 0])
        if n <= E.MICRO:
            c = min(chk.prefix_candidates(ids), key=lambda c: c[1])
            a_ids, b_ids = ids[: c[0]], ids[c[0]:]
        else:
            cands = chk.binned_candidates(ids)
            if cands:
                best = min(cands, key=lambda c: c[2])
                a_ids, b_ids = ids[best[1]], ids[~best[1]]
            else:
                a_ids, b_ids = ids[: n // 2], ids[n // 2:]
        child[me][0] = rec(a_ids, sorted_small)
        child[me][1] = rec(b_ids, sorted_small)
        return me

    root = rec(np.arange(len(tris)), False)
    assert root == 0
    lf = np.array([l[0] for l in leaves], np.int64)
    lc = np.array([l[1] for l in leaves], np.int64)
    return dict(child=np.array(child, np.int32).reshape(-1, 2), leaf_first=lf, leaf_count=lc,
                prims=np.array(prims, np.int32))


@pytest.fixture(scope="module")
def city():
    sc = scenes.prism_city(120, 300.0, 7, tx_keepout=((150.0, 150.0, 30.0),))
    return sc.tris, (150.0, 150.0, 30.0)


@pytest.mark.parametrize("alpha,dist_norm,bins", [(0.7, 1, 16), (0.4, 0, 8), (0.0, 0, 16), (1.0, 0, 32), (0.4, 2, 16)])
def test_rule_tree_passes(orc, city, alpha, dist_norm, bins):
    tris, src = city
    ex = _build(orc, tris, alpha, src, dist_norm, bins, max_leaf=2)
    st = E.check_tree(orc, tris, ex, alpha, src, dist_norm, bins)
    assert st["binned"] > 20 and st["micro"] > 100 and st["micro_roots"] > 10
    assert st["binned_exact"] == st["binned"] and st["micro_exact"] == st["micro"]


@pytest.mark.parametrize("mistake", ["mirrored_source", "raw_instead_of_scale_free", "sah_tree"])
def test_planted_mistakes_fail(orc, city, mistake):
    tris, src = city
    alpha, dn, bins = 0.4, 1, 16
    if mistake == "mirrored_source":
        ex = _build(orc, tris, alpha, (-src[0], -src[1], -src[2]), dn, bins, max_leaf=2)
    elif mistake == "raw_instead_of_scale_free":
        ex = _build(orc, tris, alpha, src, 0, bins, max_leaf=2)
    else:
        ex = _build(orc, tris, 1.0, src, dn, bins, max_leaf=2)
    with pytest.raises(AssertionError):
        E.check_tree(orc, tris, ex, alpha, src, dn, bins)


def test_node_ranges_reject_a_broken_tree(orc, city):
    tris, src = city
    ex = _build(orc, tris, 1.0, src, 0, 16, max_leaf=2)
    bad = dict(ex)
    bad["leaf_first"] = ex["leaf_first"].copy()
    bad["leaf_first"][[0, 1]] = bad["leaf_first"][[1, 0]]
    with pytest.raises(AssertionError):
        E.node_ranges(bad)


def test_slab_index_matches_float32_rule():
    # the upper end lands in the last slab, the lower end in slab 0; the scale
    # K (1 - 1e-6) / extent puts a centre exactly on a slab plane into the slab
    # below it
    c = np.array([10.0, 10.5, 12.0, 12.01, 17.999, 18.0], np.float32)
    b = E.slab_index(c, 8)
    assert b.tolist() == [0, 0, 1, 2, 7, 7]
