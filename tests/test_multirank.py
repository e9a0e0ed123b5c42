"""The benchmark's multi-rank logic on CPU with gloo, world size 2: each rank
steps its own environments (its own seed), the job time is the slowest rank's
and the job value counts every rank's env-steps. No data-path collective."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2605_19926_gb300 import inputs

    cfg = bench.shard_config(inputs.batched_keydoor_mazes(64), rank)
    t_max = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    out[rank] = (cfg["seed"], t_max, bench.job_value(world, cfg["n_envs"], 100, t_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    seeds = {out[r][0] for r in range(world)}
    assert len(seeds) == world, "each rank steps its own environments"
    for r in range(world):
        assert out[r][1] == 15.0  # the slowest rank's time
        assert out[r][2] == pytest.approx(world * 64 * 100 / 0.015)


def test_shards_generate_different_episodes(orc):
    import sys

    sys.path.insert(0, ROOT)
    import bench
    from paper_2605_19926_gb300 import inputs

    base = inputs.batched_keydoor_mazes(8)
    maps = []
    for rank in range(2):
        cfg = orc.make_config(**bench.shard_config(base, rank))
        maps.append(orc.generate(cfg, np.arange(8))["map"])
    assert (maps[0] != maps[1]).any(axis=1).all()


def test_reference_arm_prints_only_on_rank0(capsys, monkeypatch):
    import sys

    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        ref_envs, steps, warmup, gpus = 4, 1, 1, 2

    bench.run_reference(A(), {})
    assert capsys.readouterr().out == ""
