"""The multi-GPU mode is replicas only: every rank holds the whole scene and renders its own orbit
frames (no exchange step), and the bench reports the slowest rank's time over all frames.  This
runs that logic as two gloo ranks on the CPU (no GPU involved)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    frames = bench.replica_frames(rank, world, 6, 120)
    per_rank_ms = [10.0 * (rank + 1), 20.0 + 3.0 * rank]   # culled, unculled times of this rank
    job = bench.job_ms_per_frame(per_rank_ms, 6, world)
    q.put((rank, frames, job))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_split_the_orbit_and_report_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        rank, frames, job = q.get(timeout=120)
        res[rank] = (frames, job)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    f0, f1 = res[0][0], res[1][0]
    assert f0 == [0, 2, 4, 6, 8, 10] and f1 == [1, 3, 5, 7, 9, 11]
    assert not set(f0) & set(f1)
    # the slowest rank's time over all 12 frames, the same on both ranks
    expect = [20.0 / 12, 23.0 / 12]
    for r in (0, 1):
        assert res[r][1] == pytest.approx(expect)


def test_single_replica_is_plain_time_per_frame():
    import bench
    assert bench.replica_frames(0, 1, 4, 120) == [0, 1, 2, 3]
    assert bench.job_ms_per_frame([40.0, 80.0], 4, 1) == [10.0, 20.0]
