"""The multi-rank path of the benchmark (replicas, one per GPU) on CPU:
world size 2 over gloo, no GPU.  The data path has no collective; the only
exchange is the MAX of the ranks' timed regions, and the whole-job rate is
the units of all ranks over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_env()
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        mine = [12.5, 20.0][rank]                 # this rank's timed region (ms)
        t = bench.max_over_ranks(mine, dist, "cpu")
        rate = bench.job_rate(655362, w, 20, t)
        dist.barrier()
        out.put((r, w, local, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, w, local, t, rate) in enumerate(res):
        assert (r, w, local) == (rank, 2, rank)
        assert t == 20.0
        assert rate == pytest.approx(2 * 655362 * 20 / 0.020 / 1e6)


def test_single_process_needs_no_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_rate(1000, 1, 10, 1.0) == pytest.approx(10.0)


def _ref_arm(env_extra):
    import json
    import subprocess
    import sys
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    return [json.loads(l) for l in lines]


def test_reference_arm_rank0_prints_the_oracle_line_other_ranks_exit_quietly():
    (line,) = _ref_arm({"RANK": "0", "WORLD_SIZE": "2", "LOCAL_RANK": "0"})
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
    assert line["unit"] == "Mrays/s" and line["value"] > 0 and line["n_gpus"] == 2
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert _ref_arm({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
