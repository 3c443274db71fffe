"""bench.py's multi-process logic on CPU with gloo, world size 2: every rank
gets its own factor (seed offset by rank), the job's time is the slowest
rank's (max over ranks), and the reported value aggregates all ranks' work."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, w)
    G, J = bench.make_input("graded1024", seed_offset=r)
    digest = torch.tensor([float(G[0, 0]), float(G[5, 7])], dtype=torch.float64)
    gathered = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, digest)
    out[rank] = (ms, [g.tolist() for g in gathered])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, digests = res[rank]
        assert ms == pytest.approx(15.0)  # the slower rank's time, on every rank
        assert digests[0] != digests[1]   # each rank solves its own factor
