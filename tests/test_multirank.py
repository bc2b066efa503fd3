"""bench.py's replica (weak-scaling) host logic across 2 ranks on CPU (gloo)."""
import os
import socket

import numpy as np
import pytest
import torch
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
    from paper_2603_04350_gb300 import inputs as I
    p = bench.with_rank_seed(I.HEAT_DIRICHLET_1024, rank)
    local_ms = 10.0 + 5.0 * rank                     # rank 1 is the slowest
    total_ms, value = bench.aggregate(local_ms, p.unknowns, 4, world, dist, torch.device("cpu"))
    u0 = I.make_u0(p)
    f = I.make_forcing(p.with_(Nt=2))
    out[rank] = (total_ms, value, p.seed, p.n, float(f[1].sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_max_and_count_all_units():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    from paper_2603_04350_gb300 import inputs as I
    p = I.HEAT_DIRICHLET_1024
    for r in range(world):
        total_ms, value, seed, n, _ = res[r]
        assert total_ms == 15.0                                   # max over ranks
        assert value == pytest.approx(world * p.unknowns * 4 / 0.015)
        assert n == p.n
    assert res[0][2] != res[1][2] and res[0][4] != res[1][4]      # each rank its own seeded problem
