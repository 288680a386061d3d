"""The multi-GPU path of the benchmark on the CPU (gloo, world size 2): each
rank advances an independently seeded copy of the workload (weak scaling), or
its share of the batched replicas (strong scaling); no collective on the data
path; the step time is the maximum over ranks and the particle count the sum.
Launched as two spawned processes on 127.0.0.1."""
import multiprocessing as mp
import os
import socket

import numpy as np


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    systems = bench.workload("plain_sphere", rank, "fp64")
    n = float(sum(s["n"] for s in systems))
    ms, total = bench.reduce_over_ranks(dist, 1.0 + rank, n, None)
    q.put((rank, systems[0]["x"][:3].tolist(), systems[0]["params"]["seed"], ms, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_independently_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    old = os.environ.get("PYTHONPATH", "")
    os.environ["PYTHONPATH"] = root + (os.pathsep + old if old else "")
    try:
        for p in procs:
            p.start()
        out = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
        os.environ["PYTHONPATH"] = old
    assert all(p.exitcode == 0 for p in procs)
    (r0, x0, s0, ms0, n0), (r1, x1, s1, ms1, n1) = out
    assert (r0, r1) == (0, 1)
    assert s0 != s1 and not np.allclose(x0, x1)  # independent copies
    assert ms0 == ms1 == 2.0  # max over ranks
    assert n0 == n1 == 2000.0  # particles of both ranks


def _replica_worker(rank, world, port, q):
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    systems = bench.workload("replicas", rank, "mixed", nrep=24, world=world)
    n = float(sum(s["n"] for s in systems))
    _, total = bench.reduce_over_ranks(dist, 1.0, n, None)
    q.put((rank, sorted(int(s["params"]["replica"]) for s in systems), n, total,
           [int(s["n"]) for s in systems]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_the_replica_batch():
    """The batched replicas are split across the ranks (strong scaling): the
    two ranks hold disjoint sets of the same 24 replicas, together all of
    them, balanced by particle count within one replica, and the particle
    total over ranks is the batch's."""
    import bench

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    procs = [ctx.Process(target=_replica_worker, args=(r, 2, port, q)) for r in range(2)]
    old = os.environ.get("PYTHONPATH", "")
    os.environ["PYTHONPATH"] = root + (os.pathsep + old if old else "")
    try:
        for p in procs:
            p.start()
        out = sorted(q.get(timeout=300) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
        os.environ["PYTHONPATH"] = old
    assert all(p.exitcode == 0 for p in procs)
    (r0, ids0, n0, t0, sizes0), (r1, ids1, n1, t1, sizes1) = out
    assert not set(ids0) & set(ids1) and sorted(ids0 + ids1) == list(range(24))
    assert abs(n0 - n1) <= max(sizes0 + sizes1)
    assert t0 == t1 == n0 + n1
    assert bench.scaling_of("replicas") == "strong" and bench.scaling_of("ellipsoid_torus") == "weak"
