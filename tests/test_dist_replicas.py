"""The multi-GPU form of the benchmark runs independent replicas (the workloads fit one GPU;
nothing is exchanged between ranks).  Its host logic runs here on two gloo ranks on the CPU:
the job's time is the slowest rank's, its value counts every replica's site updates, and the
reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    seconds = 1.0 + rank  # rank 1 is the slow replica
    t = bench.max_over_ranks(seconds, dist, device="cpu")
    out[rank] = (t, bench.whole_job_mlups(world, 256 ** 3, 1000, t))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_replica_sets_the_time_and_all_replicas_count():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]  # every rank reports the same job figures
    t, mlups = res[0]
    assert t == 2.0
    assert mlups == pytest.approx(2 * 256 ** 3 * 1000 / 2.0 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, ref_side = 3, 3, 16

    assert bench.run_reference(Args()) == 0  # returns at once: no oracle work on rank 1
