"""The N > 1 path of bench.py on CPU with gloo (world size 2): replicas only, so the ranks
split the independent instances among themselves with no data-path collective and agree on
the job time as the maximum over ranks."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from workloads import batch_instances, serve_stream

    reqs = serve_stream(50)
    mine = bench.shard(reqs, rank, world)
    t = bench.max_over_ranks(dist, 1.0 + rank, "cpu")
    batch = bench.shard(batch_instances(16), rank, world)
    # each rank solves its own instances with the oracle (replicas: no exchange of data)
    from oracle import fmg_oracle as O
    kw = dict(batch[0], levels=2)
    lam = O.fmg_solve(O.Problem(**kw)).lam
    dist.barrier()
    out[rank] = (len(mine), [r["arrival_s"] for r in mine], t, lam, kw["zeta"])
    dist.destroy_process_group()


def test_replica_sharding_and_timing_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    from workloads import batch_instances, serve_stream
    reqs = serve_stream(50)
    n0, t0, m0, lam0, z0 = out[0]
    n1, t1, m1, lam1, z1 = out[1]
    # the shares partition the stream, keep its order, and differ by at most one
    assert n0 + n1 == len(reqs) and abs(n0 - n1) <= 1
    assert sorted(t0 + t1) == [r["arrival_s"] for r in reqs]
    # both ranks report the slowest rank's time
    assert m0 == m1 == 2.0
    # each rank solved a different instance of the batch
    assert z0 == batch_instances(16)[0]["zeta"] and z1 == batch_instances(16)[1]["zeta"]
    assert lam0 != lam1
