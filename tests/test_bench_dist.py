"""Host-side logic of bench.py's multi-rank form, run as two gloo ranks on
the CPU: the timing is the maximum over ranks, the whole-job throughput counts
every rank's work, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.setup_dist()
        assert (w, r, local) == (world, rank, rank)
        slowest = bench.max_over_ranks(times[rank], world, "cpu")
        out[rank] = slowest

        class A:
            steps, warmup = 1, 3
        if rank != 0:
            # the reference arm does nothing on ranks other than 0
            assert bench.run_reference(A, None, world, rank) == 0
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_and_throughput():
    pytest.importorskip("torch.distributed")
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    times = [12.5, 17.25]
    mp.start_processes(_rank_main, args=(world, port, times, out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1] == 17.25
    import bench
    # 2 ranks x 100 units per step x 10 steps in 17.25 ms
    assert bench.job_throughput(2, 100, 10, 17.25) == pytest.approx(2 * 100 * 10 / 0.01725)
