"""The bench's N > 1 path on CPU: two `gloo` ranks (replicas only, no data-path collective).
Each rank's job time enters once through a MAX all-reduce, the whole-job rate counts every
rank's units, and the reference arm runs on rank 0 alone."""
import argparse
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms_by_rank, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_max = bench.slowest_rank_ms(ms_by_rank[rank], world)
        rate = bench.replica_rate(1.0e9, 5, world, ms_max)
        # the reference arm: only rank 0 runs (and prints); the others return at once
        ref_rc = bench.run_reference(argparse.Namespace(workload="doppler_1e5", gpus=world, steps=1, warmup=0,
                                                        ref_step_s=0.05)) if rank != 0 else None
        out[rank] = (ms_max, rate, ref_rc)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_rank():
    world, port = 2, _free_port()
    ms_by_rank = [12.5, 40.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, ms_by_rank, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms_max, rate, ref_rc = res[rank]
        assert ms_max == 40.0
        assert rate == pytest.approx(world * 1.0e9 * 5 / 0.040)
    assert res[1][2] == 0


def test_single_rank_needs_no_process_group():
    assert bench.slowest_rank_ms(7.0, 1) == 7.0
    assert bench.replica_rate(100.0, 2, 1, 1000.0) == pytest.approx(200.0)
