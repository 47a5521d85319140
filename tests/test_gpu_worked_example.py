"""The device build on the hand-worked Eq. 2 example (Sec. II.B): four unit
triangles on a line, source at the origin.  The root split the device picks
must be the one derived by hand for each alpha, with the raw distance term
and with the scale-free one (reading c2), where the choice flips between
alpha = 0.4 and 0.5 (needs a GB300)."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def rb():
    from paper_2208_10008_gb300 import rtbvh
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    rtbvh.lib()
    return rtbvh


def _root_left_size(e):
    def size(c):
        if c < 0:
            return int(e["leaf_count"][-1 - c])
        return size(e["child"][c][0]) + size(e["child"][c][1])
    return size(e["child"][0][0])


def test_device_root_split_is_the_hand_derived_one(rb):
    g = json.load(open(os.path.join(GOLDEN, "eq2_worked_example.json")))
    tris = np.asarray(g["tris"], np.float32)
    cases = [(0, a, i) for a, i in g["best_split"].items()]
    cases += [(1, a, i) for a, i in g["dist_norm_1"]["best_split"].items()]
    cases += [(2, a, i) for a, i in g["dist_norm_2"]["best_split"].items()]
    for dist_norm, alpha_s, i_best in cases:
        s = rb.rt_scene_upload(tris)
        rb.rt_bvh_build(s, alpha=float(alpha_s), source=(0.0, 0.0, 0.0), max_leaf=1, dist_norm=dist_norm)
        e = rb.rt_bvh_export(s)
        assert e["info"]["status"] == 0 and len(e["child"]) == 3
        assert sorted(e["prims"].tolist()) == [0, 1, 2, 3]
        assert _root_left_size(e) == i_best, (dist_norm, alpha_s)
        s.destroy()
