"""The N > 1 benchmark path on CPU: two gloo ranks.

`bench.py --gpus N` runs one independent flow per rank (replicas: the
parameter points shard with no exchange) and reports the whole job as the
evaluations of all ranks over the slowest rank's time.  These tests run that
reduction, the reference arm's rank gating and the rendezvous on two CPU
processes with the gloo backend."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, local = bench.dist_init()
    # rank r timed 10 + r ms for 100 (r + 1) evaluations
    ms, ev = bench.reduce_over_ranks(10.0 + rank, 100 * (rank + 1))
    # the reference arm: ranks other than 0 leave at once without work
    rc_ref = bench.run_reference(type("A", (), {"warmup": 3, "steps": 1})()) if rank else None
    dist.barrier()
    out[rank] = (w, r, local, ms, ev, rc_ref)
    dist.destroy_process_group()


def test_two_rank_replica_reduction_and_reference_gating():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        w, r, local, ms, ev, rc_ref = res[rank]
        assert (w, r, local) == (world, rank, rank)
        assert ms == 11.0            # slowest rank
        assert ev == 100.0 + 200.0   # all ranks' evaluations
    assert res[1][5] == 0


def test_single_process_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(7.5, 42) == (7.5, 42.0)
