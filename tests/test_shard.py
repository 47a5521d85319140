"""Ray sharding over ranks (one process per GPU): the ranges and the gather,
on CPU with world size 2 over gloo.  Each rank computes its range with the
float64 checker standing in for its GPU; the gathered hits must equal the
single-process result bit for bit."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_ranges_are_balanced_disjoint_and_cover():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2208_10008_gb300.shard import ray_range
    for n in (0, 1, 7, 8, 655362, 1 << 21):
        for world in (1, 2, 3, 8):
            rs = [ray_range(n, k, world) for k in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[k][1] == rs[k + 1][0] for k in range(world - 1))
            sizes = [hi - lo for lo, hi in rs]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        ray_range(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import oracle
    from paper_2208_10008_gb300 import scenes
    from paper_2208_10008_gb300.shard import gather_ranges, ray_range
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        sc, rays, _ = scenes.workload_tiny()
        rays = rays[:4001]                      # an odd count: ranges of unequal size
        lo, hi = ray_range(len(rays), rank, ws)
        h = oracle.closest_brute(sc.tris, rays[lo:hi])
        local = torch.from_numpy(np.stack([h.t.astype(np.float32), h.id.view(np.float32)], 1).copy())
        full = gather_ranges(local, len(rays))
        dist.barrier()
        out.put((rank, (lo, hi), full.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gather_the_single_rank_result():
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2208_10008_gb300 import scenes
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc, rays, _ = scenes.workload_tiny()
    rays = rays[:4001]
    h = oracle.closest_brute(sc.tris, rays)
    ref = np.stack([h.t.astype(np.float32), h.id.view(np.float32)], 1)
    assert res[0][1] == (0, 2001) and res[1][1] == (2001, 4001)
    for _, _, full in res:                      # every rank holds the whole, identical result
        assert np.array_equal(full.view(np.uint32), ref.view(np.uint32))


@pytest.mark.gpu
def test_sharded_trace_on_one_gpu_equals_the_plain_call():
    # the module's GPU path with a one-rank NCCL group (the only group one GPU
    # allows): its range is every ray, the gather returns them all
    import sys
    sys.path.insert(0, ROOT)
    from paper_2208_10008_gb300 import rtbvh, scenes
    from paper_2208_10008_gb300.shard import trace_closest_sharded
    assert torch.cuda.is_available()
    sc, rays, p = scenes.workload_medium(level=6)
    s = rtbvh.rt_scene_upload(sc.tris)
    rtbvh.rt_bvh_build(s, alpha=0.7, source=p["source"], dist_norm=1)
    r = torch.from_numpy(rays).cuda()
    dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % _free_port(), rank=0, world_size=1)
    try:
        full = trace_closest_sharded(s, r)
        mine, (lo, hi) = trace_closest_sharded(s, r, gather=False)
        ref = rtbvh.rt_trace_closest(s, r)
        torch.cuda.synchronize()
        assert (lo, hi) == (0, len(rays))
        assert torch.equal(full.view(torch.int32), ref.view(torch.int32))
        assert torch.equal(mine.view(torch.int32), ref.view(torch.int32))
    finally:
        dist.destroy_process_group()
