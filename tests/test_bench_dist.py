"""The multi-GPU bench path on CPU: two gloo ranks shard the frames with no data
exchange, and the job's time is the slowest rank's (max over ranks)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        frames = bench.shard_frames(rank, 4)
        mine = 10.0 + 5.0 * rank                  # rank 1 is the slow one
        dist.barrier()
        ms = bench.max_over_ranks(mine, ws, "cpu")
        out.put((rank, frames, ms, bench.whole_job_rate(ws, 100, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, f0, ms0, v0), (r1, f1, ms1, v1) = res
    assert set(f0).isdisjoint(f1) and sorted(f0 + f1) == list(range(8))
    assert ms0 == ms1 == 15.0                      # both ranks report the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 100 / 0.015)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.shard_frames(0, 3) == [0, 1, 2]
    assert bench.whole_job_rate(1, 10, 100.0) == pytest.approx(100.0)
