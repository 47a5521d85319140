"""The batched city at full size (10,000 prisms, 200,742 triangles; 16
transmitters, 13.1M Fibonacci rays; needs a GB300): one run of the batched
pipeline with one reflection order, and seeded samples of its direct and
reflected rays compared with the float64 brute force over every triangle.
The reflected rays are the device's own (float32) rays, each with the
triangle it leaves from skipped, as the checker's input."""
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


def test_batched_city_samples_match_checker(rb, orc):
    sc, tx, counts, rx = scenes.workload_batched()
    assert sc.n_tri == 200_742 and int(counts.sum()) == 13_108_520
    s = rb.rt_scene_upload(sc.tris)
    rb.rt_bvh_build(s, alpha=0.7, dist_norm=1, source=tuple(tx.mean(0)), max_leaf=4, bins=16)
    b = rb.Batch(s, tx, counts, rb.RT_RAYS_FIBONACCI, max_order=1, tmax=1000.0)
    b.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(33)

    rays0, hits0, _, n0 = b.order(0)
    assert n0 == int(counts.sum())
    i0 = torch.from_numpy(np.sort(rng.choice(n0, 16384, replace=False))).cuda()
    r0, h0 = rays0[i0].cpu().numpy(), hits0[i0].cpu().numpy()
    compare_closest(h0, orc.closest_brute(sc.tris, r0), sc.tris, r0, "batched city, direct rays")

    rays1, hits1, src1, n1 = b.order(1)
    assert 0 < n1 < n0
    i1 = torch.from_numpy(np.sort(rng.choice(n1, min(8192, n1), replace=False))).cuda()
    r1, h1 = rays1[i1].cpu().numpy(), hits1[i1].cpu().numpy()
    parent = src1[i1].long()
    _, skip, _, _ = split_hits(hits0[parent].cpu().numpy())   # the triangle each bounce leaves from
    assert (skip >= 0).all()
    compare_closest(h1, orc.closest_brute(sc.tris, r1, skip=skip), sc.tris, r1, "batched city, first bounce")
    b.destroy()
    s.destroy()
