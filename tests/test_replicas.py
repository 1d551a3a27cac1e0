"""Replica sharding of independent points (host logic, CPU only).

Two gloo ranks each take their longest-first share of a mixed-D_cut sample of
the (beta, Delta) grid, produce a per-point result, and gather: every point
must come back exactly once, the shares must be balanced, and every rank must
compute the same partition without communicating."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2609_20536_b300 import replicas
from paper_2609_20536_b300.workloads import grid_points


def sample():
    pts = grid_points()
    return [pts[(i * 61) % len(pts)] for i in range(96)]


def test_shard_partitions_and_balances():
    pts = sample()
    for world in (1, 2, 3, 4):
        parts = [replicas.shard(pts, world, r) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(pts)))
        ld = replicas.loads(pts, world)
        assert max(ld) <= 1.05 * min(ld)  # LPT over 96 points of four sizes
    with pytest.raises(ValueError):
        replicas.shard(pts, 2, 2)


def test_cost_model_follows_the_step_sizes():
    # D0 = 9: the first step fuses 9 x 9 legs, later steps run at D_cut
    assert replicas.step_sizes(4, 64, 3) == [(9, 9), (9, 64), (64, 64)]
    assert replicas.point_cost(4, 64, 25) > replicas.point_cost(4, 24, 25) > 0


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pts = sample()
    mine = replicas.shard(pts, world, rank)
    results = {i: (rank, round(pts[i].beta * 1000 + pts[i].delta, 9)) for i in mine}
    merged = replicas.gather(results)
    if rank == 0:
        with open(os.path.join(out_dir, "merged.txt"), "w") as f:
            for k in sorted(merged):
                f.write(f"{k} {merged[k][0]} {merged[k][1]}\n")
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_gather_every_point_once(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    lines = open(tmp_path / "merged.txt").read().split("\n")[:-1]
    pts = sample()
    assert len(lines) == len(pts)
    owners = {}
    for ln in lines:
        k, r, v = ln.split()
        k, r = int(k), int(r)
        owners[k] = r
        assert abs(float(v) - (pts[k].beta * 1000 + pts[k].delta)) < 1e-6
    for r in range(world):
        assert sorted(k for k, o in owners.items() if o == r) == replicas.shard(pts, world, r)
