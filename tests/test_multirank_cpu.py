"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas), each
solving its own image, the job time is the slowest rank's and the value
counts every rank's outer iterations."""
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
    from synth import CONFIGS
    spec = bench.replica_spec(CONFIGS["C5"], rank, world)
    local_ms = 1000.0 * (rank + 1)               # rank 1 is the slow one
    ms_max = bench.max_over_ranks_dist(local_ms, world, "cpu")
    dist.barrier()
    out[rank] = (spec.seed, ms_max, bench.job_seconds_per_outer(ms_max, 4, world))
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_time():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    seeds = {out[r][0] for r in range(world)}
    assert len(seeds) == world                   # independent images
    for r in range(world):
        assert out[r][1] == 2000.0               # max over ranks
        assert out[r][2] == pytest.approx(2000.0 / 1e3 / (4 * world))
